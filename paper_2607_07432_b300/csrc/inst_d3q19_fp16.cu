// Kernel instantiation for D3Q19 with __half storage and float arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d3q19_fp16() { return Engine<lbmib::D3Q19, __half, float>::ops(); }
}  // namespace lbmib_host
