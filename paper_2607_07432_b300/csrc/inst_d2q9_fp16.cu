// Kernel instantiation for D2Q9 with __half storage and float arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d2q9_fp16() { return Engine<lbmib::D2Q9, __half, float>::ops(); }
}  // namespace lbmib_host
