// Network tile kernels (network.cu): declarations shared with the step driver.
#pragma once
#include "gnep_internal.h"

namespace gnep {

constexpr int kNetBlocks = 456;  // persistent blocks of the backward pass (3 per SM)

// Species-homogeneous tiles over the species-grouped atom order.
struct Tiles {
  const int* perm;
  int soff[9];
  int tbase[9];  // first tile of each species; tbase[ns] = tile count
  int ns;
};

Tiles make_tiles(const gnep_nlist* nl, int ns, int tile_atoms);

template <int D, int HP, int NS, int NQR, int KR>
int mlp_setup();
template <int D, int HP, int NS, int NQR, int KR>
int mlp_forward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st);
template <int D, int HP>
int mlp_backward(const gnep_model* m, gnep_nlist* nl, cudaStream_t st);

// Hidden width padded to the instantiated tile width.
inline int hidden_pad(int H) { return H <= 32 ? 32 : H <= 64 ? 64 : 128; }

// Tensor-core network (network_tc.cu): BF16 (TF32 = false) or TF32 operands,
// FP32 accumulation; hidden width padded to a multiple of 16 up to 112.
constexpr int kMaxHiddenTc = 112;
inline int hidden_pad_tc(int H) { return H <= 32 ? 32 : H <= 64 ? 64 : 112; }
template <bool TF32, int D, int HPn, int NS, int NQR, int KR>
int mlp_setup_tc();
template <bool TF32, int D, int HPn, int NS, int NQR, int KR>
int mlp_forward_tc(const gnep_model* m, gnep_nlist* nl, cudaStream_t st);
template <bool TF32, int D, int HPn>
int mlp_backward_tc(const gnep_model* m, gnep_nlist* nl, cudaStream_t st);
// One block of the tensor-core kernels' bounded-wait protocol on an mbarrier
// that nothing arrives on (raises TIMEOUT in the model's error flag).
int wait_selftest(const gnep_model* m, uint64_t limit_ns, cudaStream_t st);

}  // namespace gnep
