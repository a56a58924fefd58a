// Warp-level tensor-core products for the per-atom contractions of the angular
// sweeps: mma.sync m16n8k8 with TF32 operands and FP32 accumulation.
//
// Fragment layout for lane l, g = l / 4, t = l % 4 (PTX ISA, matrix fragments
// of mma.m16n8k8 with .tf32):
//   A (16 x 8, row major)  a0 (g, t)   a1 (g+8, t)   a2 (g, t+4)   a3 (g+8, t+4)
//   B (8 x 8, col major)   b0 (t, g)   b1 (t+4, g)
//   C (16 x 8)             c0 (g, 2t)  c1 (g, 2t+1)  c2 (g+8, 2t)  c3 (g+8, 2t+1)
//
// A product with SPLIT carries each operand x as hi = rna_tf32(x) and
// lo = rna_tf32(x - hi) and accumulates lo*hi + hi*lo + hi*hi; the dropped
// lo*lo term is below FP32 rounding (the split-operand method of Ootomo and
// Yokota, 2022).  The hi*hi terms and the two correction terms go to separate
// accumulators that are added once at the end: folding the corrections into
// the running sum, whose low bits the tensor core's accumulation drops, made
// the error of a K = 16 dot product 1.7 times that of an FP32 FMA chain, while
// two chains match it (measured on random operands of mixed sign).  Without
// SPLIT a product takes the operands' TF32 truncations alone (TF32 accuracy).
#pragma once
#include <cstdint>

namespace gnep {

struct FragA {
  uint32_t h[4], l[4];
};
struct FragB {
  uint32_t h[2], l[2];
};

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// With SPLIT: hi rounded to nearest, lo the rounded remainder.  Without: the
// FP32 bits as they are (the tensor core reads a TF32 operand from the upper 19
// bits, i.e. rounds toward zero), which saves the conversion where single TF32
// products are accurate enough anyway.
template <bool SPLIT>
__device__ __forceinline__ void split_tf32(float x, uint32_t& h, uint32_t& l) {
  if constexpr (SPLIT) {
    h = tf32_rna(x);
    l = tf32_rna(x - __uint_as_float(h));
  } else {
    h = __float_as_uint(x);
    l = 0u;
  }
}

template <bool SPLIT>
__device__ __forceinline__ void frag_a(FragA& a, float a0, float a1, float a2, float a3) {
  split_tf32<SPLIT>(a0, a.h[0], a.l[0]);
  split_tf32<SPLIT>(a1, a.h[1], a.l[1]);
  split_tf32<SPLIT>(a2, a.h[2], a.l[2]);
  split_tf32<SPLIT>(a3, a.h[3], a.l[3]);
}

template <bool SPLIT>
__device__ __forceinline__ void frag_b(FragB& b, float b0, float b1) {
  split_tf32<SPLIT>(b0, b.h[0], b.l[0]);
  split_tf32<SPLIT>(b1, b.h[1], b.l[1]);
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A C fragment (16 x 8, FP32): hi*hi chain v and, with SPLIT, correction chain c.
template <bool SPLIT>
struct Acc {
  float v[4];
  float c[SPLIT ? 4 : 1];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = 0.f;
#pragma unroll
    for (int r = 0; r < (SPLIT ? 4 : 1); ++r) c[r] = 0.f;
  }
  __device__ __forceinline__ float get(int r) const {
    if constexpr (SPLIT) return v[r] + c[r];
    return v[r];
  }
};

// d += A B.
template <bool SPLIT>
__device__ __forceinline__ void mma_acc(Acc<SPLIT>& d, const FragA& a, const FragB& b) {
  if constexpr (SPLIT) {
    mma_tf32(d.c, a.l, b.h);
    mma_tf32(d.c, a.h, b.l);
  }
  mma_tf32(d.v, a.h, b.h);
}

}  // namespace gnep
