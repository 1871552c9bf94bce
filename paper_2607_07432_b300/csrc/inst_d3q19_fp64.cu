// Kernel instantiation for D3Q19 with double storage and double arithmetic.
#include "engine.cuh"

namespace lbmib_host {
const Ops* ops_d3q19_fp64() { return Engine<lbmib::D3Q19, double, double>::ops(); }
}  // namespace lbmib_host
