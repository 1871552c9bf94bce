// Kernel instantiation for D3Q19 with __nv_bfloat16 storage and float arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d3q19_bf16() { return Engine<lbmib::D3Q19, __nv_bfloat16, float>::ops(); }
}  // namespace lbmib_host
