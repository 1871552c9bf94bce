// Kernel instantiation for D2Q9 with double storage and double arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d2q9_fp64() { return Engine<lbmib::D2Q9, double, double>::ops(); }
}  // namespace lbmib_host
