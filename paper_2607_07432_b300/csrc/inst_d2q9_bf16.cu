// Kernel instantiation for D2Q9 with __nv_bfloat16 storage and float arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d2q9_bf16() { return Engine<lbmib::D2Q9, __nv_bfloat16, float>::ops(); }
}  // namespace lbmib_host
