// Angular sweeps for l_max > 4 (sweeps_lmax.cu): the terms l = 5..8 of Eq. 7
// (App. B, B5-B8).  Each call launches one kernel on `st`; the arrays are those
// of the workspace, with S rows of (l_max + 1)^2 - 1 components.
#pragma once
#include <cuda_runtime.h>

#include "gnep_internal.h"

namespace gnep {

template <class C>
int hi_setup();
// sweep 1: S_nlm (Sout) and the angular descriptor columns of G
template <class C>
int hi_desc_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, float* S, float* G);
// sweep 2: the angular pair forces dE_i/dr_ij into dA
template <class C>
int hi_force_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, const float* S, const float* Ep,
                     float4* dA);
// sweep 3: Sdot, the angular columns of Gdot and the tangent directions w_ij
template <class C>
int hi_tangent_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, const float4* a, const float* Bs,
                       const float* S, float* Sd, float* Gd, float4* wij);
// sweep 4: the angular part of dL/dc into cpart[block][c^R + c^A] for nb blocks
template <class C>
int hi_cgrad_angular(const gnep_model* m, const gnep_nlist* nl, cudaStream_t st, int nb, const float4* wij,
                     const float* S, const float* Sd, const float* Gb, const float* Ep, float* cpart);

}  // namespace gnep
