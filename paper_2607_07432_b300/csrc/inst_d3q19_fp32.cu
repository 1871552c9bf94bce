// Kernel instantiation for D3Q19 with float storage and float arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d3q19_fp32() { return Engine<lbmib::D3Q19, float, float>::ops(); }
}  // namespace lbmib_host
