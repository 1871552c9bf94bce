// Kernel instantiation for D2Q9 with float storage and float arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d2q9_fp32() { return Engine<lbmib::D2Q9, float, float>::ops(); }
}  // namespace lbmib_host
