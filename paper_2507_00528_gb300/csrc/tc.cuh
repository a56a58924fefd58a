// Fifth-generation tensor-core primitives (tcgen05, sm_100a family) as inline
// PTX: tensor-memory allocation, shared-memory matrix descriptors, MMA issue,
// completion through an mbarrier with a bounded wait, and TMEM loads.
//
// Operand layout (both A and B "K-major", no swizzle): a matrix of R rows and
// C columns (C along the contraction K) is stored as 8-row x 16-byte core
// matrices.  Element (r, c) sits at byte
//     (r / 8) * SBO + (c / EPC) * LBO + (r % 8) * 16 + (c % EPC) * ES,
// with ES the element size, EPC = 16 / ES elements per core row and
// SBO = (C / EPC) * LBO the stride between 8-row groups; core matrices adjacent
// along K are LBO bytes apart (the descriptor's leading-dimension offset): 128
// packs them, 144 leaves 16 bytes after each, which puts the core matrices
// that one warp's row-wise or transposed element stores touch 4 banks apart.
// The two operands of one MMA may take different LBOs (each has its own
// descriptor); mma_chain takes one for both, so operands contracted with each
// other share it.
// One MMA of M = 128 consumes 32 bytes of K (16 BF16 or 8 TF32 elements) and
// accumulates D[m][n] += sum_k A[m][k] B[n][k] in FP32 in tensor memory, row m
// in TMEM lane m, column n in TMEM column n.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace gnep {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <bool TF32>
struct Elem;
template <>
struct Elem<false> {  // BF16 operands, kind::f16
  static constexpr int ES = 2, EPC = 8, KSTEP = 16, FMT = 1;
};
template <>
struct Elem<true> {  // TF32 operands, kind::tf32
  static constexpr int ES = 4, EPC = 4, KSTEP = 8, FMT = 2;
};

// Byte stride between 8-row groups of an operand with C columns.
template <bool TF32>
__host__ __device__ constexpr uint32_t sbo(int C, uint32_t lbo = 128u) {
  return (uint32_t)(C / Elem<TF32>::EPC) * lbo;
}

template <bool TF32>
__device__ __forceinline__ uint32_t core_off(int r, int c, uint32_t sbo_, uint32_t lbo = 128u) {
  constexpr int ES = Elem<TF32>::ES, EPC = Elem<TF32>::EPC;
  return (uint32_t)(r >> 3) * sbo_ + (uint32_t)(c / EPC) * lbo + (uint32_t)(r & 7) * 16u + (uint32_t)(c % EPC) * ES;
}

// FP32 -> operand bits (round to nearest).
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ uint16_t to_bf16(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// Store one element.
template <bool TF32>
__device__ __forceinline__ void st_elem(uint8_t* base, uint32_t off, float x) {
  if constexpr (TF32)
    *reinterpret_cast<uint32_t*>(base + off) = to_tf32(x);
  else
    *reinterpret_cast<uint16_t*>(base + off) = to_bf16(x);
}

// Store one 4-byte word: 4 / ES consecutive columns of one row (the first at a
// column divisible by 4 / ES).
template <bool TF32>
__device__ __forceinline__ void st_word(uint8_t* base, uint32_t off, const float (&x)[4 / Elem<TF32>::ES]) {
  if constexpr (TF32)
    *reinterpret_cast<uint32_t*>(base + off) = to_tf32(x[0]);
  else
    *reinterpret_cast<uint32_t*>(base + off) = (uint32_t)to_bf16(x[0]) | ((uint32_t)to_bf16(x[1]) << 16);
}

// Store one 16-byte core row: EPC consecutive columns c0.. of row r (c0 % EPC == 0).
template <bool TF32>
__device__ __forceinline__ void st_chunk(uint8_t* base, uint32_t off, const float* v) {
  uint4 u;
  if constexpr (TF32) {
    u = make_uint4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
  } else {
    auto p = [](float a, float b) { return (uint32_t)to_bf16(a) | ((uint32_t)to_bf16(b) << 16); };
    u = make_uint4(p(v[0], v[1]), p(v[2], v[3]), p(v[4], v[5]), p(v[6], v[7]));
  }
  *reinterpret_cast<uint4*>(base + off) = u;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row group) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo_) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo_ >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format FMT, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if constexpr (TF32)
    asm volatile("{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;}" ::"r"(
                     d_tmem), "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile("{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}" ::"r"(
                     d_tmem), "l"(a), "l"(b), "r"(id), "r"(acc));
}

// D (M = 128 rows, N columns at d_tmem) (+)= A [128 x K] . B [N x K]^T, both
// operands K-major in shared memory with the given 8-row-group strides.
template <bool TF32>
__device__ __forceinline__ void mma_chain(uint32_t d_tmem, const void* A, uint32_t a_sbo, const void* B, uint32_t b_sbo,
                                          int K, int N, bool accumulate, uint32_t lbo = 128u) {
  using E = Elem<TF32>;
  const uint32_t id = idesc(E::FMT, 128, N);
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
  for (int k = 0; k < K; k += E::KSTEP) {
    const uint32_t koff = (uint32_t)(k / E::EPC) * lbo;
    mma<TF32>(d_tmem, sdesc(a0 + koff, lbo, a_sbo), sdesc(b0 + koff, lbo, b_sbo), id,
              (accumulate || k > 0) ? 1u : 0u);
  }
}

// Arrive on the mbarrier once all MMAs issued so far by this thread have completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;");
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the given phase of the mbarrier; gives up after limit_ns and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase, uint64_t limit_ns) {
  const uint32_t a = smem_u32(mbar);
  uint32_t done = 0;
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    asm volatile("{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p;}"
                 : "=r"(done)
                 : "r"(a), "r"(phase));
    if (done) return true;
    if ((it & 255u) == 0) {
      const uint64_t t = globaltimer();
      if (it == 0)
        t0 = t;
      else if (t - t0 > limit_ns)
        return false;
    }
  }
}

// Tensor-memory allocation (one warp), its release and the allocation permit.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32w..32w+31).
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  // the wait names the registers so that no use of them is scheduled before it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

constexpr int pow2_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }

}  // namespace tc
}  // namespace gnep
