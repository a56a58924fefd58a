// Neighbour sets of Eq. 2: N^i = { (j, n) : |r_j + n.H - r_i| < r_c, (j, n) != (i, 0) }
// over every periodic image n, for the radial (r_c^R) and angular (r_c^A)
// cut-offs, in canonical order (j ascending, then image shift lexicographic).
//
// The accept/reject decision is that of FP64 with explicitly rounded operations
// (no fused multiply-add) in the fixed order
//   s = (na a + nb b) + nc c,  d = (r_j + s) - r_i,  d2 = (dx^2 + dy^2) + dz^2,
// so the list equals that of any plain FP64 evaluation of the same expression.
// FP64 arithmetic is slow on this GPU, so candidates are first measured in
// FP32; only those whose FP32 d2 lies within a relative 2e-3 of a cut-off (far
// above the FP32 error of d2 for coordinates below 10^4 A) take the FP64 test.
// The stored r_ij is formed in float-float arithmetic (about 44 bits) and
// rounded to FP32.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "gnep_internal.h"

namespace gnep {

namespace {

// Structures with more atoms than this take the binned search, the others
// the all-pairs one (the two give identical lists).
constexpr int kCellMinAtoms = 1024;


__global__ void k_atom_struct(const int* __restrict__ off, int S, int N, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int lo = 0, hi = S - 1;
  while (lo < hi) {  // last s with off[s] <= i
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  out[i] = lo;
}

// Images needed per cell direction: floor(rc / w) + 1, w = V / |b x c| etc.
// tw[s][x] = rc / w_x bounds |df_x + n_x| for any pair within rc.  Also the
// inverse cell (FP64), the cell split into FP32 high and low parts, and the
// bins of the binned search: nbin[s][x] = floor(w_x / (rc / 2)) bins along
// direction x (at least 1), reduced until the structure has no more bins than
// atoms (so that the bins of structure s can be numbered from its first atom
// index on).
__global__ void k_image_range(const double* __restrict__ cell, int S, double rc, const int* __restrict__ soff,
                              int* __restrict__ kr, float* __restrict__ tw, double* __restrict__ hinv,
                              float* __restrict__ hsplit, int* __restrict__ nbin, int* __restrict__ big) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double* H = cell + 9 * s;
  const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                     H[2] * (H[3] * H[7] - H[4] * H[6]);
  const double id = 1.0 / det;
  const double inv[9] = {(H[4] * H[8] - H[5] * H[7]) * id, (H[2] * H[7] - H[1] * H[8]) * id,
                         (H[1] * H[5] - H[2] * H[4]) * id, (H[5] * H[6] - H[3] * H[8]) * id,
                         (H[0] * H[8] - H[2] * H[6]) * id, (H[2] * H[3] - H[0] * H[5]) * id,
                         (H[3] * H[7] - H[4] * H[6]) * id, (H[1] * H[6] - H[0] * H[7]) * id,
                         (H[0] * H[4] - H[1] * H[3]) * id};
  for (int q = 0; q < 9; ++q) {
    hinv[9 * s + q] = inv[q];
    const float hi = (float)H[q];
    hsplit[18 * s + q] = hi;
    hsplit[18 * s + 9 + q] = (float)(H[q] - (double)hi);
  }
  const double* a = cell + 9 * s;
  const double* b = a + 3;
  const double* c = a + 6;
  const double bc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
  const double ca[3] = {c[1] * a[2] - c[2] * a[1], c[2] * a[0] - c[0] * a[2], c[0] * a[1] - c[1] * a[0]};
  const double ab[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
  const double vol = fabs(a[0] * bc[0] + a[1] * bc[1] + a[2] * bc[2]);
  const double n[3] = {norm3d(bc[0], bc[1], bc[2]), norm3d(ca[0], ca[1], ca[2]), norm3d(ab[0], ab[1], ab[2])};
  int nb[3];
  for (int x = 0; x < 3; ++x) {
    kr[3 * s + x] = (int)floor(rc / (vol / n[x])) + 1;
    tw[3 * s + x] = (float)(rc / (vol / n[x]));
    const double q = floor((vol / n[x]) / (0.5 * rc));
    nb[x] = q < 1.0 ? 1 : q > 64.0 ? 64 : (int)q;
  }
  const int cap = max(1, soff[s + 1] - soff[s]);
  if (cap > kCellMinAtoms) atomicOr(big, 1);  // some structure takes the binned search
  while (nb[0] * nb[1] * nb[2] > cap) {  // at most 189 steps
    const int x = (nb[0] >= nb[1] && nb[0] >= nb[2]) ? 0 : (nb[1] >= nb[2] ? 1 : 2);
    --nb[x];
  }
  for (int x = 0; x < 3; ++x) nbin[3 * s + x] = nb[x];
}

// Bin of atom i of structure s in the binned search (from its FP32 fractional
// coordinates; any consistent assignment is valid, since the search visits
// every bin that can hold a neighbour and the lists are sorted afterwards).
__device__ __forceinline__ int atom_bin(float4 f, const int* nb) {
  const int bx = min(nb[0] - 1, max(0, (int)floorf(f.x * (float)nb[0])));
  const int by = min(nb[1] - 1, max(0, (int)floorf(f.y * (float)nb[1])));
  const int bz = min(nb[2] - 1, max(0, (int)floorf(f.z * (float)nb[2])));
  return bx + nb[0] * (by + nb[1] * bz);
}

// Atoms per bin (bins of structure s are numbered from its first atom index).
__global__ void k_bin_count(int N, const int* __restrict__ atom_struct, const int* __restrict__ soff,
                            const int* __restrict__ nbin, const float4* __restrict__ frac, const int* __restrict__ big,
                            int* __restrict__ bcount) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || *big == 0) return;
  const int s = atom_struct[i];
  if (soff[s + 1] - soff[s] <= kCellMinAtoms) return;  // searched without bins
  atomicAdd(&bcount[soff[s] + atom_bin(frac[i], nbin + 3 * s)], 1);
}

// Atom indices by bin, at the scanned bin starts (the order inside a bin is
// free: it only sets the order in which candidates are tested).
__global__ void k_bin_fill(int N, const int* __restrict__ atom_struct, const int* __restrict__ soff,
                           const int* __restrict__ nbin, const float4* __restrict__ frac,
                           const long long* __restrict__ bstart, const int* __restrict__ big, int* __restrict__ bcursor,
                           int* __restrict__ batom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N || *big == 0) return;
  const int s = atom_struct[i];
  if (soff[s + 1] - soff[s] <= kCellMinAtoms) return;  // searched without bins
  const int b = soff[s] + atom_bin(frac[i], nbin + 3 * s);
  batom[bstart[b] + atomicAdd(&bcursor[b], 1)] = i;
}

// Per atom: fractional coordinates f = r H^-1 (FP32; only used to bound image
// shifts, and checked to lie in [0, 1)), and the position split into FP32
// high and low parts (w of the high part carries the species).
__global__ void k_atom_prep(int N, const int* __restrict__ atom_struct, const double* __restrict__ pos,
                            const int* __restrict__ type, const double* __restrict__ hinv,
                            float4* __restrict__ frac, float4* __restrict__ phi, float4* __restrict__ plo,
                            int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* inv = hinv + 9 * atom_struct[i];
  const double* p = pos + 3 * (size_t)i;
  double f[3];
  bool wrapped = true;
  for (int x = 0; x < 3; ++x) {
    f[x] = p[0] * inv[x] + p[1] * inv[3 + x] + p[2] * inv[6 + x];
    wrapped = wrapped && f[x] > -1e-9 && f[x] < 1.0 + 1e-9;
  }
  if (!wrapped) atomicOr(err, kErrUnwrapped);
  frac[i] = make_float4((float)f[0], (float)f[1], (float)f[2], 0.f);
  const float hx = (float)p[0], hy = (float)p[1], hz = (float)p[2];
  phi[i] = make_float4(hx, hy, hz, (float)type[i]);
  plo[i] = make_float4((float)(p[0] - (double)hx), (float)(p[1] - (double)hy), (float)(p[2] - (double)hz), 0.f);
}

// Error-free transformations for float-float arithmetic.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// r_j + n.H - r_i in float-float (about 44 significant bits), rounded to FP32.
__device__ __forceinline__ float pair_component(float pjh, float pjl, float pih, float pil, int na, int nb, int nc,
                                                float ah, float al, float bh, float bl, float ch, float cl) {
  float h, e, t, u;
  two_sum(pjh, -pih, h, e);
  float lo = e + (pjl - pil);
  two_prod((float)na, ah, t, u);
  lo += u + (float)na * al;
  two_sum(h, t, h, e);
  lo += e;
  two_prod((float)nb, bh, t, u);
  lo += u + (float)nb * bl;
  two_sum(h, t, h, e);
  lo += e;
  two_prod((float)nc, ch, t, u);
  lo += u + (float)nc * cl;
  two_sum(h, t, h, e);
  lo += e;
  return h + lo;
}

__device__ __forceinline__ double pair_d2_exact(const double* H, const double* pi, const double* pj,
                                                int na, int nb, int nc, double d[3]) {
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const double s = __dadd_rn(__dadd_rn(__dmul_rn((double)na, H[x]), __dmul_rn((double)nb, H[3 + x])),
                               __dmul_rn((double)nc, H[6 + x]));
    d[x] = __dsub_rn(__dadd_rn(pj[x], s), pi[x]);
  }
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

struct ListParams {
  double rc2[2];     // exact squared cut-offs (radial, angular)
  float lo2[2];      // FP32 d2 below: inside (FP32 decision)
  float hi2[2];      // FP32 d2 above: outside (FP32 decision)
  float reject2;     // max(hi2): candidates above it are outside both
};

// The list decisions for neighbour j of atom i at image n (na, nb, nc) of
// structure s: FP32 away from the cut-offs, the exact FP64 expression within
// the band.  dj = phi_j - phi_i (high parts), Hh the FP32 high parts of the
// cell.  Both searches (all pairs, binned) take their decisions here.
__device__ __forceinline__ void decide_pair(int i, int j, int na, int nb, int nc, const float (&dj)[3],
                                            const float (&Hh)[9], const ListParams& lp,
                                            const double* __restrict__ cell, const double* __restrict__ pos, int s,
                                            bool& in0, bool& in1) {
  in0 = in1 = false;
  if (j == i && na == 0 && nb == 0 && nc == 0) return;
  const float fx = dj[0] + ((float)na * Hh[0] + (float)nb * Hh[3] + (float)nc * Hh[6]);
  const float fy = dj[1] + ((float)na * Hh[1] + (float)nb * Hh[4] + (float)nc * Hh[7]);
  const float fz = dj[2] + ((float)na * Hh[2] + (float)nb * Hh[5] + (float)nc * Hh[8]);
  const float d2f = fx * fx + fy * fy + fz * fz;
  if (d2f > lp.reject2) return;
  in0 = d2f < lp.lo2[0];
  in1 = d2f < lp.lo2[1];
  const bool band0 = !in0 && d2f <= lp.hi2[0], band1 = !in1 && d2f <= lp.hi2[1];
  if (band0 || band1) {  // near a cut-off: the FP64 decision
    const double* Hd = cell + 9 * s;
    const double H[9] = {Hd[0], Hd[1], Hd[2], Hd[3], Hd[4], Hd[5], Hd[6], Hd[7], Hd[8]};
    const double pi[3] = {pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]};
    const double pj[3] = {pos[3 * (size_t)j], pos[3 * (size_t)j + 1], pos[3 * (size_t)j + 2]};
    double d[3];
    const double d2 = pair_d2_exact(H, pi, pj, na, nb, nc, d);
    if (band0) in0 = d2 < lp.rc2[0];
    if (band1) in1 = d2 < lp.rc2[1];
  }
}

// Per-atom slots of the slot passes: the first cap[L] entries of atom i's
// list L go to j[L][i cap[L] + k], sh[L][...]; k_compact moves them into the
// CSR lists once the counts are scanned.
struct Slots {
  int cap[2];
  int* j[2];
  char4* sh[2];
};

// One warp per central atom i.  Lane l tests the neighbours j = a0 + l,
// a0 + l + 32, ...: in each round of 32 consecutive j every lane walks the
// images of its j in lexicographic order, and the warp places the accepted
// entries by an exclusive scan of the per-lane counts, so each list comes out
// in canonical order (j ascending, then image), written into the CSR lists at
// the offsets that the slot pass counted: the writing pass of a batch in which
// some atom has more entries than its slots hold.  It takes the slot passes'
// decisions (FP32 away from the cut-offs, FP64 within the band).  A lane
// keeps up to kBuf accepted images of its j in a packed register; a round in
// which some lane accepts more walks the images again to place them.
constexpr int kBuf = 4;

__global__ void __launch_bounds__(128) k_pairs(
    int N, const int* __restrict__ struct_off, const int* __restrict__ atom_struct,
    const double* __restrict__ pos, const double* __restrict__ cell, const int* __restrict__ krange,
    const float* __restrict__ tw, const float* __restrict__ hsplit, const float4* __restrict__ frac,
    const float4* __restrict__ phi, const float4* __restrict__ plo, ListParams lp,
    const long long* __restrict__ off0, const long long* __restrict__ off1, int* __restrict__ j0,
    int* __restrict__ own0, float4* __restrict__ r0, char4* __restrict__ sh0, int* __restrict__ j1,
    int* __restrict__ own1, float4* __restrict__ r1, char4* __restrict__ sh1) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= N) return;  // the whole warp
  const int s = atom_struct[i];
  const int a0 = struct_off[s], a1 = struct_off[s + 1];
  float Hh[9], Hl[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    Hh[q] = hsplit[18 * s + q];
    Hl[q] = hsplit[18 * s + 9 + q];
  }
  const float4 pih = phi[i], pil = plo[i];
  const int ka = krange[3 * s], kb = krange[3 * s + 1], kc = krange[3 * s + 2];
  const bool packable = ka <= 7 && kb <= 7 && kc <= 7;  // image indices fit 4 bits
  // |r_j + n.H - r_i| >= |df_x + n_x| w_x, so only shifts with |df_x + n_x| < rc / w_x
  // (with a margin far above FP32 rounding) can pass the test below.
  const float4 fi = frac[i];
  const float t0 = tw[3 * s] + 1e-3f, t1 = tw[3 * s + 1] + 1e-3f, t2 = tw[3 * s + 2] + 1e-3f;
  int base0 = 0, base1 = 0;
  for (int jb = a0; jb < a1; jb += 32) {
    const int j = jb + lane;
    const bool vj = j < a1;
    const float4 pjh = vj ? phi[j] : pih;
    const float4 fj = vj ? frac[j] : fi;
    const float dj[3] = {pjh.x - pih.x, pjh.y - pih.y, pjh.z - pih.z};
    const float dfa = fj.x - fi.x, dfb = fj.y - fi.y, dfc = fj.z - fi.z;
    const int alo = max(-ka, (int)ceilf(-t0 - dfa)), ahi = vj ? min(ka, (int)floorf(t0 - dfa)) : alo - 1;
    const int blo = max(-kb, (int)ceilf(-t1 - dfb)), bhi = min(kb, (int)floorf(t1 - dfb));
    const int clo = max(-kc, (int)ceilf(-t2 - dfc)), chi = min(kc, (int)floorf(t2 - dfc));
    // the list decisions for image n of this lane's j
    auto decide = [&](int na, int nb, int nc, bool& in0, bool& in1) {
      decide_pair(i, j, na, nb, nc, dj, Hh, lp, cell, pos, s, in0, in1);
    };
    // places one accepted entry at the next positions of its lists
    auto put = [&](int na, int nb, int nc, bool in0, bool in1, int& w0, int& w1) {
      const char4 sv = make_char4((signed char)na, (signed char)nb, (signed char)nc, 0);
      const float4 pjl = plo[j];
      const float rx = pair_component(pjh.x, pjl.x, pih.x, pil.x, na, nb, nc, Hh[0], Hl[0], Hh[3], Hl[3], Hh[6], Hl[6]);
      const float ry = pair_component(pjh.y, pjl.y, pih.y, pil.y, na, nb, nc, Hh[1], Hl[1], Hh[4], Hl[4], Hh[7], Hl[7]);
      const float rz = pair_component(pjh.z, pjl.z, pih.z, pil.z, na, nb, nc, Hh[2], Hl[2], Hh[5], Hl[5], Hh[8], Hl[8]);
      const float4 rv = make_float4(rx, ry, rz, pjh.w);
      if (in0) { const long long d = off0[i] + w0; j0[d] = j; own0[d] = i; r0[d] = rv; sh0[d] = sv; }
      if (in1) { const long long d = off1[i] + w1; j1[d] = j; own1[d] = i; r1[d] = rv; sh1[d] = sv; }
      w0 += in0;
      w1 += in1;
    };
    int n0 = 0, n1 = 0, nacc = 0;
    unsigned long long buf = 0;
    for (int na = alo; na <= ahi; ++na)
      for (int nb = blo; nb <= bhi; ++nb)
        for (int nc = clo; nc <= chi; ++nc) {
          bool in0, in1;
          decide(na, nb, nc, in0, in1);
          if (!in0 && !in1) continue;
          if (packable && nacc < kBuf)
            buf |= (unsigned long long)((na + 8) | (nb + 8) << 4 | (nc + 8) << 8 | (int)in0 << 12 | (int)in1 << 13)
                   << (16 * nacc);
          ++nacc;
          n0 += in0;
          n1 += in1;
        }
    int p0 = n0, p1 = n1;  // inclusive scan over the lanes (j order)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u0 = __shfl_up_sync(0xffffffffu, p0, o), u1 = __shfl_up_sync(0xffffffffu, p1, o);
      if (lane >= o) {
        p0 += u0;
        p1 += u1;
      }
    }
    const int tot0 = __shfl_sync(0xffffffffu, p0, 31), tot1 = __shfl_sync(0xffffffffu, p1, 31);
    int w0 = base0 + p0 - n0, w1 = base1 + p1 - n1;
    if (!__any_sync(0xffffffffu, nacc > kBuf || (nacc > 0 && !packable))) {
      for (int e = 0; e < nacc; ++e) {
        const int v = (int)((buf >> (16 * e)) & 0xffffu);
        put((v & 15) - 8, ((v >> 4) & 15) - 8, ((v >> 8) & 15) - 8, (v >> 12) & 1, (v >> 13) & 1, w0, w1);
      }
    } else {  // walk the images again, placing each accepted one
      for (int na = alo; na <= ahi; ++na)
        for (int nb = blo; nb <= bhi; ++nb)
          for (int nc = clo; nc <= chi; ++nc) {
            bool in0, in1;
            decide(na, nb, nc, in0, in1);
            if (in0 || in1) put(na, nb, nc, in0, in1, w0, w1);
          }
    }
    base0 += tot0;
    base1 += tot1;
  }
}

// The slot pass for structures of at most kCellMinAtoms atoms, one warp per
// central atom i, with the candidates flattened: in each round of kFlatJ = 64
// consecutive j (two per lane) the lanes count the images their j may have
// within the cut-offs (the fractional bounds of k_pairs), a warp scan lays
// those (j, image) candidates out in canonical order (j ascending, then image
// lexicographic) and the lanes then take them 32 at a time, so that every lane
// tests a candidate in every step instead of walking its own j's images while
// the others wait.  The round's per-j bounds and scan sit in the warp's shared
// memory; each lane finds its candidate's j by a binary search over the scan.
// Accepted entries are placed by ballots in the same canonical order (counts
// exact; the first cap entries of each list go to the atom's slots).  Two j per
// lane fill about half of the candidate steps' lanes on cells of the
// 32-400-atom workload, where one j per lane filled under a third.
constexpr int kFlatWarps = 4, kFlatJ = 64;

__global__ void __launch_bounds__(32 * kFlatWarps) k_pairs_flat(
    int N, const int* __restrict__ struct_off, const int* __restrict__ atom_struct,
    const double* __restrict__ pos, const double* __restrict__ cell, const int* __restrict__ krange,
    const float* __restrict__ tw, const float* __restrict__ hsplit, const float4* __restrict__ frac,
    const float4* __restrict__ phi, ListParams lp, int* __restrict__ cnt0, int* __restrict__ cnt1, Slots sl) {
  // per warp and round: dj = phi_j - phi_i, (alo, blo, clo, j), (nb count, nc
  // count, candidates before this j) and the inclusive candidate counts
  __shared__ float4 sdj[kFlatWarps][kFlatJ];
  __shared__ int4 slo[kFlatWarps][kFlatJ];
  __shared__ int4 scnt[kFlatWarps][kFlatJ];
  __shared__ int sincl[kFlatWarps][kFlatJ];
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  if (i >= N) return;  // the whole warp
  const int s = atom_struct[i];
  const int a0 = struct_off[s], a1 = struct_off[s + 1];
  if (a1 - a0 > kCellMinAtoms) return;  // the binned search takes this structure
  float Hh[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) Hh[q] = hsplit[18 * s + q];
  const float4 pih = phi[i];
  const int ka = krange[3 * s], kb = krange[3 * s + 1], kc = krange[3 * s + 2];
  const float4 fi = frac[i];
  const float t0 = tw[3 * s] + 1e-3f, t1 = tw[3 * s + 1] + 1e-3f, t2 = tw[3 * s + 2] + 1e-3f;
  const unsigned lt = (1u << lane) - 1u;
  int w0 = 0, w1 = 0;  // entries of each list so far (warp-uniform)
  for (int jb = a0; jb < a1; jb += kFlatJ) {
    int base = 0;  // candidates of the round's first half (after its scan)
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // j = jb + 32 h + lane at position 32 h + lane
      const int j = jb + 32 * h + lane;
      const bool vj = j < a1;
      const float4 pjh = vj ? phi[j] : pih;
      const float4 fj = vj ? frac[j] : fi;
      const float dfa = fj.x - fi.x, dfb = fj.y - fi.y, dfc = fj.z - fi.z;
      const int alo = max(-ka, (int)ceilf(-t0 - dfa)), ahi = vj ? min(ka, (int)floorf(t0 - dfa)) : alo - 1;
      const int blo = max(-kb, (int)ceilf(-t1 - dfb)), bhi = min(kb, (int)floorf(t1 - dfb));
      const int clo = max(-kc, (int)ceilf(-t2 - dfc)), chi = min(kc, (int)floorf(t2 - dfc));
      const int nbc = max(0, bhi - blo + 1), ncc = max(0, chi - clo + 1);
      const int ncand = max(0, ahi - alo + 1) * nbc * ncc;  // this j's candidate images
      int incl = ncand;  // inclusive scan over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      incl += base;
      const int x = 32 * h + lane;
      sdj[wb][x] = make_float4(pjh.x - pih.x, pjh.y - pih.y, pjh.z - pih.z, 0.f);
      slo[wb][x] = make_int4(alo, blo, clo, j);
      scnt[wb][x] = make_int4(nbc, ncc, incl - ncand, 0);
      sincl[wb][x] = incl;
      base = __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const int total = base;
    for (int cb = 0; cb < total; cb += 32) {
      const int c = cb + lane;
      const bool valid = c < total;
      int L = 0;  // the position whose j owns candidate c: incl[L - 1] <= c < incl[L] (at most 63)
#pragma unroll
      for (int st = kFlatJ / 2; st >= 1; st >>= 1)
        if (sincl[wb][L + st - 1] <= c) L += st;
      bool in0 = false, in1 = false;
      int na = 0, nb = 0, nc = 0, oj = 0;
      if (valid) {  // image m of the owner's (na, nb, nc) ranges, nc fastest (a few steps: no division)
        const float4 d4 = sdj[wb][L];
        const int4 lo = slo[wb][L], cn = scnt[wb][L];
        const float odj[3] = {d4.x, d4.y, d4.z};
        oj = lo.w;
        int r = c - cn.z;
        const int bc = cn.x * cn.y;
        na = lo.x;
        while (r >= bc) {
          r -= bc;
          ++na;
        }
        nb = lo.y;
        while (r >= cn.y) {
          r -= cn.y;
          ++nb;
        }
        nc = lo.z + r;
        decide_pair(i, oj, na, nb, nc, odj, Hh, lp, cell, pos, s, in0, in1);
      }
      const unsigned b0 = __ballot_sync(0xffffffffu, in0), b1 = __ballot_sync(0xffffffffu, in1);
      const char4 sv = make_char4((signed char)na, (signed char)nb, (signed char)nc, 0);
      if (in0) {
        const int w = w0 + __popc(b0 & lt);
        if (w < sl.cap[0]) {
          const size_t q = (size_t)i * sl.cap[0] + w;
          sl.j[0][q] = oj;
          sl.sh[0][q] = sv;
        }
      }
      if (in1) {
        const int w = w1 + __popc(b1 & lt);
        if (w < sl.cap[1]) {
          const size_t q = (size_t)i * sl.cap[1] + w;
          sl.j[1][q] = oj;
          sl.sh[1][q] = sv;
        }
      }
      w0 += __popc(b0);
      w1 += __popc(b1);
    }
    __syncwarp();  // the round's shared entries are read before the next round writes them
  }
  if (lane == 0) {
    cnt0[i] = w0;
    cnt1[i] = w1;
  }
}

// Binned search, one warp per central atom i (the slot pass) of the
// structures above kCellMinAtoms atoms; the smaller ones take the all-pairs
// search (k_pairs_flat), which is as fast there: at cell widths below 3 r_c the
// visited bins cover about the whole cell.  The bins of structure s split its
// cell into nbin[s] parts along each cell direction; every (j, n) within r_c of
// i has f_j + n inside (f_i - t, f_i + t) along each direction (t = r_c / w_x,
// with a margin), i.e. in one of the extended bins floor((f_i - t) nbin) ..
// floor((f_i + t) nbin), so the warp visits those bins (lane per bin; extended
// bin B holds the atoms of bin B mod nbin at the image floor(B / nbin)) and
// tests their atoms with the same decision as the all-pairs search.  Accepted
// entries collect in shared memory as keys (j, image, lists); each entry's
// position in each list is its rank among the list's entries in canonical
// order (j ascending, then image lexicographic), so the slots hold exactly the
// lists of the all-pairs search.  Counts are exact even when an atom overflows
// its slots (the writing pass then takes the batch).
constexpr int kCellWarps = 4;
constexpr int kCellBuf = 160;  // accepted entries a warp ranks per atom (both lists)

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__global__ void __launch_bounds__(32 * kCellWarps) k_pairs_cell(
    int N, const int* __restrict__ struct_off, const int* __restrict__ atom_struct,
    const double* __restrict__ pos, const double* __restrict__ cell, const float* __restrict__ tw,
    const float* __restrict__ hsplit, const int* __restrict__ nbin, const long long* __restrict__ bstart,
    const int* __restrict__ batom, const float4* __restrict__ frac, const float4* __restrict__ phi, ListParams lp,
    const int* __restrict__ big, int* __restrict__ cnt0, int* __restrict__ cnt1, Slots sl) {
  if (*big == 0) return;  // no structure of this batch takes the binned search
  __shared__ unsigned long long key[kCellWarps][kCellBuf];
  __shared__ int nacc[kCellWarps], nin[kCellWarps][2];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warps stride over the atoms (a small grid: most batches have no structure
  // for this search, and then it ends after one pass of cheap tests)
  for (int i = blockIdx.x * kCellWarps + w; i < N; i += gridDim.x * kCellWarps) {
    const int s = atom_struct[i], a0 = struct_off[s];
    if (struct_off[s + 1] - a0 <= kCellMinAtoms) continue;  // taken by the all-pairs search
    if (lane == 0) {
      nacc[w] = 0;
      nin[w][0] = nin[w][1] = 0;
    }
    __syncwarp();
    const long long Q0 = bstart[a0];
    float Hh[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Hh[q] = hsplit[18 * s + q];
    const float4 pih = phi[i], fi = frac[i];
    const float f[3] = {fi.x, fi.y, fi.z};
    int nb[3], lo[3], cnt[3];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      nb[x] = nbin[3 * s + x];
      const float t = tw[3 * s + x] + 2e-3f;
      lo[x] = (int)floorf((f[x] - t) * (float)nb[x]);
      cnt[x] = (int)floorf((f[x] + t) * (float)nb[x]) - lo[x] + 1;
    }
    const int NB = cnt[0] * cnt[1] * cnt[2];
    for (int e = lane; e < NB; e += 32) {
      const int B[3] = {lo[0] + e % cnt[0], lo[1] + (e / cnt[0]) % cnt[1], lo[2] + e / (cnt[0] * cnt[1])};
      int n[3], bx[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        n[x] = floor_div(B[x], nb[x]);
        bx[x] = B[x] - n[x] * nb[x];
      }
      const int bin = bx[0] + nb[0] * (bx[1] + nb[1] * bx[2]);
      const int q0 = (int)(bstart[a0 + bin] - Q0), q1 = (int)(bstart[a0 + bin + 1] - Q0);
      for (int q = q0; q < q1; ++q) {
        const int j = batom[Q0 + q];
        const float4 pjh = phi[j];
        const float dj[3] = {pjh.x - pih.x, pjh.y - pih.y, pjh.z - pih.z};
        bool in0, in1;
        decide_pair(i, j, n[0], n[1], n[2], dj, Hh, lp, cell, pos, s, in0, in1);
        if (!in0 && !in1) continue;
        if (in0) atomicAdd(&nin[w][0], 1);
        if (in1) atomicAdd(&nin[w][1], 1);
        const int slot = atomicAdd(&nacc[w], 1);
        if (slot < kCellBuf)
          key[w][slot] = ((unsigned long long)j << 26) | ((unsigned long long)(n[0] + 128) << 18) |
                         ((unsigned long long)(n[1] + 128) << 10) | ((unsigned long long)(n[2] + 128) << 2) |
                         ((unsigned long long)in1 << 1) | (unsigned long long)in0;
      }
    }
    __syncwarp();
    const int M = nacc[w], c0 = nin[w][0], c1 = nin[w][1];
    if (lane == 0) {
      cnt0[i] = c0;
      cnt1[i] = c1;
    }
    if (M <= kCellBuf && c0 <= sl.cap[0] && c1 <= sl.cap[1]) {  // else the writing pass takes the batch
      for (int e = lane; e < M; e += 32) {
        const unsigned long long ke = key[w][e];
        int r0 = 0, r1 = 0;
        for (int e2 = 0; e2 < M; ++e2) {  // keys are distinct: ranks are positions
          const unsigned long long k2 = key[w][e2];
          const bool lt = k2 < ke;
          r0 += (lt && (k2 & 1ull)) ? 1 : 0;
          r1 += (lt && (k2 & 2ull)) ? 1 : 0;
        }
        const int j = (int)(ke >> 26);
        const char4 sv = make_char4((signed char)((int)((ke >> 18) & 255ull) - 128),
                                    (signed char)((int)((ke >> 10) & 255ull) - 128),
                                    (signed char)((int)((ke >> 2) & 255ull) - 128), 0);
        if (ke & 1ull) {
          const size_t q = (size_t)i * sl.cap[0] + r0;
          sl.j[0][q] = j;
          sl.sh[0][q] = sv;
        }
        if (ke & 2ull) {
          const size_t q = (size_t)i * sl.cap[1] + r1;
          sl.j[1][q] = j;
          sl.sh[1][q] = sv;
        }
      }
    }
    __syncwarp();  // the keys are read before the next atom's entries replace them
  }
}

// Copies the per-atom slots of both lists into the CSR lists and forms r_ij,
// one warp per atom: the atom's cell, position and offsets are read once per
// warp and the lanes take its entries (the float-float arithmetic runs on
// dense lanes).
__global__ void __launch_bounds__(256) k_compact(int N, Slots sl, const int* __restrict__ cnt0,
                                                 const int* __restrict__ cnt1, const long long* __restrict__ off0,
                                                 const long long* __restrict__ off1,
                                                 const int* __restrict__ atom_struct, const float* __restrict__ hsplit,
                                                 const float4* __restrict__ phi, const float4* __restrict__ plo,
                                                 int* __restrict__ j0, int* __restrict__ own0, float4* __restrict__ r0,
                                                 char4* __restrict__ sh0, int* __restrict__ j1, int* __restrict__ own1,
                                                 float4* __restrict__ r1, char4* __restrict__ sh1) {
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= N) return;  // the whole warp
  const float* Hs = hsplit + 18 * atom_struct[i];
  float H[18];
#pragma unroll
  for (int q = 0; q < 18; ++q) H[q] = Hs[q];
  const float4 pih = phi[i], pil = plo[i];
  // the lanes run over the radial entries and then the angular ones as one range
  const int n0 = cnt0[i], n1 = cnt1[i];  // at most the slots (the writing pass takes the batch otherwise)
  const long long d00 = off0[i], d01 = off1[i];
  for (int e = lane; e < n0 + n1; e += 32) {
    const int L = e >= n0 ? 1 : 0, c = L ? e - n0 : e;
    int* jo = L ? j1 : j0;
    int* ow = L ? own1 : own0;
    float4* ro = L ? r1 : r0;
    char4* so = L ? sh1 : sh0;
    {
      const size_t g = (size_t)i * (L ? sl.cap[1] : sl.cap[0]) + c;
      const long long d = (L ? d01 : d00) + c;
      const int jj = (L ? sl.j[1] : sl.j[0])[g];
      const char4 sv = (L ? sl.sh[1] : sl.sh[0])[g];
      const float4 pjh = phi[jj], pjl = plo[jj];
      const int na = sv.x, nb = sv.y, nc = sv.z;
      const float rx = pair_component(pjh.x, pjl.x, pih.x, pil.x, na, nb, nc, H[0], H[9], H[3], H[12], H[6], H[15]);
      const float ry = pair_component(pjh.y, pjl.y, pih.y, pil.y, na, nb, nc, H[1], H[10], H[4], H[13], H[7], H[16]);
      const float rz = pair_component(pjh.z, pjl.z, pih.z, pil.z, na, nb, nc, H[2], H[11], H[5], H[14], H[8], H[17]);
      jo[d] = jj;
      ow[d] = i;
      ro[d] = make_float4(rx, ry, rz, pjh.w);
      so[d] = sv;
    }
  }
}

// Exclusive scan of int counts into int64 offsets: one block per 1024 items,
// then the block totals, recursively.
__global__ void k_scan_block(const long long* __restrict__ in, const int* __restrict__ in32, int64_t n,
                             long long* __restrict__ out, long long* __restrict__ block_sums) {
  __shared__ long long sh[1024];
  const int64_t g = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  long long v = 0;
  if (g < n) v = in32 ? (long long)in32[g] : in[g];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    long long t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (g < n) out[g] = sh[threadIdx.x] - v;
  if (threadIdx.x == 1023) block_sums[blockIdx.x] = sh[1023];
}

__global__ void k_scan_add(long long* __restrict__ out, int64_t n, const long long* __restrict__ add) {
  const int64_t g = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  if (g < n) out[g] += add[blockIdx.x];
}

// Largest neighbour count per list (integer maxima: order-free).
__global__ void k_max2(int N, const int* __restrict__ c0, const int* __restrict__ c1, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int a = i < N ? c0[i] : 0, b = i < N ? c1[i] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], a);
    atomicMax(&out[1], b);
  }
}

constexpr int kSlotsRadial = 96;   // per-atom slots of the one-pass build (radial list)
constexpr int kSlotsAngular = 32;  // (angular list)

__global__ void k_to_int(const long long* __restrict__ in, int64_t n, int* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[g] = (int)in[g];
}

// Reverse pair: the entry (i, -n) in j's list, found by binary search on the
// canonical key (j, na, nb, nc).
__global__ void k_reverse(int64_t P, const int* __restrict__ off, const int* __restrict__ jj,
                          const int* __restrict__ own, const char4* __restrict__ sh,
                          int* __restrict__ rev, int* __restrict__ err) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int i = own[p], j = jj[p];
  const char4 s = sh[p];
  const int key[4] = {i, -s.x, -s.y, -s.z};
  int lo = off[j], hi = off[j + 1] - 1, found = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const char4 t = sh[mid];
    const int cand[4] = {jj[mid], t.x, t.y, t.z};
    int cmp = 0;
    for (int q = 0; q < 4 && cmp == 0; ++q) cmp = (cand[q] < key[q]) ? -1 : (cand[q] > key[q]) ? 1 : 0;
    if (cmp == 0) { found = mid; break; }
    if (cmp < 0) lo = mid + 1; else hi = mid - 1;
  }
  if (found < 0) { atomicOr(err, kErrRevMissing); found = (int)p; }
  rev[p] = found;
}

// Exclusive scan of in (int32 when in32 is set, else int64) into out.
int scan_rec(const long long* in64, const int* in32, int64_t n, long long* out,
             std::vector<void*>& tmp, cudaStream_t st) {
  const int64_t nb = (n + 1023) / 1024;
  long long* sums = nullptr;
  GNEP_CUDA(cudaMallocAsync(&sums, sizeof(long long) * (nb + 1), st));
  tmp.push_back(sums);
  k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(in64, in32, n, out, sums);
  GNEP_CHECK_LAUNCH("k_scan_block");
  if (nb > 1) {
    long long* scanned = nullptr;
    GNEP_CUDA(cudaMallocAsync(&scanned, sizeof(long long) * (nb + 1), st));
    tmp.push_back(scanned);
    const int rc = scan_rec(sums, nullptr, nb, scanned, tmp, st);
    if (rc) return rc;
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(out, n, scanned);
    GNEP_CHECK_LAUNCH("k_scan_add");
  }
  return GNEP_OK;
}

}  // namespace

int build_lists(gnep_model* m, gnep_nlist* nl, cudaStream_t st) {
  const int N = nl->n_atoms, S = nl->n_struct;
  std::vector<void*> tmp;
  auto cleanup = [&]() {
    for (auto p : tmp) cudaFreeAsync(p, st);
  };
  int *cnt = nullptr, *kr = nullptr, *bins = nullptr;
  float *tw = nullptr, *hsplit = nullptr;
  double* hinv = nullptr;
  float4 *frac = nullptr, *phi = nullptr, *plo = nullptr;
  long long* offs = nullptr;
  GNEP_CUDA(cudaMallocAsync(&cnt, sizeof(int) * 2 * (size_t)(N + 1), st));
  GNEP_CUDA(cudaMallocAsync(&kr, sizeof(int) * 3 * (size_t)S, st));
  GNEP_CUDA(cudaMallocAsync(&offs, sizeof(long long) * 2 * (size_t)(N + 1), st));
  GNEP_CUDA(cudaMallocAsync(&tw, sizeof(float) * 3 * (size_t)S, st));
  GNEP_CUDA(cudaMallocAsync(&hsplit, sizeof(float) * 18 * (size_t)S, st));
  GNEP_CUDA(cudaMallocAsync(&hinv, sizeof(double) * 9 * (size_t)S, st));
  GNEP_CUDA(cudaMallocAsync(&frac, sizeof(float4) * 3 * (size_t)N, st));
  phi = frac + N;
  plo = frac + 2 * (size_t)N;
  // bins: nbin [3 S], counts and cursors [N + 1] each, atoms by bin [N]
  GNEP_CUDA(cudaMallocAsync(&bins, sizeof(int) * (3 * (size_t)S + 3 * (size_t)N + 3), st));
  int* nbin = bins;
  int* bcount = bins + 3 * (size_t)S;
  int* bcursor = bcount + (N + 1);
  int* big = bcursor + (N + 1);  // set when some structure takes the binned search
  int* batom = big + 1;
  for (void* p : {(void*)cnt, (void*)kr, (void*)tw, (void*)hsplit, (void*)hinv, (void*)frac, (void*)offs, (void*)bins})
    tmp.push_back(p);
  GNEP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (size_t)(N + 1), st));
  GNEP_CUDA(cudaMemsetAsync(bcount, 0, sizeof(int) * (2 * (size_t)(N + 1) + 1), st));  // and bcursor, big

  k_atom_struct<<<blocks_for(N, 256), 256, 0, st>>>(nl->struct_off, S, N, nl->atom_struct);
  const double rcmax = nl->rcr > nl->rca ? nl->rcr : nl->rca;
  k_image_range<<<blocks_for(S, 128), 128, 0, st>>>(nl->cell, S, rcmax, nl->struct_off, kr, tw, hinv, hsplit, nbin,
                                                     big);
  k_atom_prep<<<blocks_for(N, 256), 256, 0, st>>>(N, nl->atom_struct, nl->pos, nl->type, hinv, frac, phi, plo,
                                                   m->err);
  GNEP_CHECK_LAUNCH("k_image_range");
  // atoms by bin
  long long* bstart = nullptr;
  GNEP_CUDA(cudaMallocAsync(&bstart, sizeof(long long) * (size_t)(N + 1), st));
  tmp.push_back(bstart);
  k_bin_count<<<blocks_for(N, 256), 256, 0, st>>>(N, nl->atom_struct, nl->struct_off, nbin, frac, big, bcount);
  if (int rc = scan_rec(nullptr, bcount, N + 1, bstart, tmp, st)) {
    cleanup();
    return rc;
  }
  k_bin_fill<<<blocks_for(N, 256), 256, 0, st>>>(N, nl->atom_struct, nl->struct_off, nbin, frac, bstart, big,
                                                  bcursor, batom);
  GNEP_CHECK_LAUNCH("k_bin_fill");

  ListParams lp;
  lp.rc2[0] = nl->rcr * nl->rcr;
  lp.rc2[1] = nl->rca * nl->rca;
  for (int L = 0; L < 2; ++L) {
    lp.lo2[L] = (float)(lp.rc2[L] * (1.0 - 2e-3));
    lp.hi2[L] = (float)(lp.rc2[L] * (1.0 + 2e-3));
  }
  lp.reject2 = lp.hi2[0] > lp.hi2[1] ? lp.hi2[0] : lp.hi2[1];

  int* cnt0 = cnt;
  int* cnt1 = cnt + (N + 1);
  // one pass into per-atom slots (cap entries per atom and list); atoms with
  // more neighbours than that fall back to a second, writing pass
  Slots sl;
  sl.cap[0] = kSlotsRadial;
  sl.cap[1] = kSlotsAngular;
  {
    const size_t n0 = (size_t)N * sl.cap[0], n1 = (size_t)N * sl.cap[1];
    char* slots = nullptr;
    GNEP_CUDA(cudaMallocAsync(&slots, (n0 + n1) * (sizeof(int) + sizeof(char4)), st));
    tmp.push_back(slots);
    sl.j[0] = reinterpret_cast<int*>(slots);
    sl.j[1] = sl.j[0] + n0;
    sl.sh[0] = reinterpret_cast<char4*>(sl.j[1] + n1);
    sl.sh[1] = sl.sh[0] + n0;
  }
  k_pairs_flat<<<blocks_for((int64_t)N * 32, 32 * kFlatWarps), 32 * kFlatWarps, 0, st>>>(N, nl->struct_off, nl->atom_struct, nl->pos,
                                                                 nl->cell, kr, tw, hsplit, frac, phi, lp, cnt0, cnt1,
                                                                 sl);
  k_pairs_cell<<<(unsigned)std::min<int64_t>((N + kCellWarps - 1) / kCellWarps, 1216), 32 * kCellWarps, 0, st>>>(
      N, nl->struct_off, nl->atom_struct, nl->pos, nl->cell, tw, hsplit, nbin, bstart, batom, frac, phi, lp, big,
      cnt0, cnt1, sl);
  GNEP_CHECK_LAUNCH("pair search");
  int* maxc = nullptr;
  GNEP_CUDA(cudaMallocAsync(&maxc, sizeof(int) * 2, st));
  tmp.push_back(maxc);
  GNEP_CUDA(cudaMemsetAsync(maxc, 0, sizeof(int) * 2, st));
  k_max2<<<blocks_for(N, 256), 256, 0, st>>>(N, cnt0, cnt1, maxc);

  long long* off0 = offs;
  long long* off1 = offs + (N + 1);
  int rc = scan_rec(nullptr, cnt0, N + 1, off0, tmp, st);
  if (rc) { cleanup(); return rc; }
  rc = scan_rec(nullptr, cnt1, N + 1, off1, tmp, st);
  if (rc) { cleanup(); return rc; }
  long long tot[2];
  int hmax[2] = {0, 0};
  GNEP_CUDA(cudaMemcpyAsync(&tot[0], off0 + N, sizeof(long long), cudaMemcpyDeviceToHost, st));
  GNEP_CUDA(cudaMemcpyAsync(&tot[1], off1 + N, sizeof(long long), cudaMemcpyDeviceToHost, st));
  GNEP_CUDA(cudaMemcpyAsync(hmax, maxc, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  int herr = 0;
  GNEP_CUDA(cudaMemcpyAsync(&herr, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  // the angular offsets come back with the counts: the host cuts the angular
  // tiles from them while the lists are compacted on the device
  if (nl->host_aoff_cap < (int64_t)N + 1) {
    if (nl->host_aoff) cudaFreeHost(nl->host_aoff);
    nl->host_aoff = nullptr;
    nl->host_aoff_cap = 0;
    GNEP_CUDA(cudaMallocHost(&nl->host_aoff, sizeof(long long) * ((size_t)N + 1)));
    nl->host_aoff_cap = (int64_t)N + 1;
  }
  nl->host_aoff_n = (int64_t)N + 1;
  GNEP_CUDA(cudaMemcpyAsync(nl->host_aoff, off1, sizeof(long long) * ((size_t)N + 1), cudaMemcpyDeviceToHost, st));
  GNEP_CUDA(cudaStreamSynchronize(st));
  if (herr & kErrUnwrapped) {
    cleanup();
    GNEP_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), st));
    return set_error(GNEP_ERR_INVALID_ARG, "positions must be wrapped into their cell (fractional coordinates in [0,1))");
  }
  for (int L = 0; L < 2; ++L)
    if (tot[L] >= (1LL << 31) - 1) {
      cleanup();
      return set_error(GNEP_ERR_NEIGHBOR_OVERFLOW, "pair count exceeds 32-bit indices; split the batch");
    }

  for (int L = 0; L < 2; ++L) {
    PairList& P = nl->L[L];
    if (tot[L] > P.cap) {
      cudaFree(P.j); cudaFree(P.owner); cudaFree(P.rev); cudaFree(P.rij); cudaFree(P.shift);
      const int64_t cap = tot[L] > 0 ? tot[L] + tot[L] / 8 + 64 : 64;  // headroom for rebuilds (MD)
      GNEP_CUDA(cudaMalloc(&P.j, sizeof(int) * cap));
      GNEP_CUDA(cudaMalloc(&P.owner, sizeof(int) * cap));
      if (L == 1) GNEP_CUDA(cudaMalloc(&P.rev, sizeof(int) * cap));  // the force sweep pairs angular entries
      GNEP_CUDA(cudaMalloc(&P.rij, sizeof(float4) * cap));
      GNEP_CUDA(cudaMalloc(&P.shift, sizeof(char4) * cap));
      P.cap = cap;
    }
    if (!P.off) GNEP_CUDA(cudaMalloc(&P.off, sizeof(int) * (size_t)(N + 1)));
    P.n = tot[L];
    k_to_int<<<blocks_for(N + 1, 256), 256, 0, st>>>(L == 0 ? off0 : off1, N + 1, P.off);
  }
  if (hmax[0] <= sl.cap[0] && hmax[1] <= sl.cap[1]) {
    if (N > 0)
      k_compact<<<blocks_for((int64_t)N * 32, 256), 256, 0, st>>>(
          N, sl, cnt0, cnt1, off0, off1, nl->atom_struct, hsplit, phi, plo, nl->L[0].j, nl->L[0].owner,
          nl->L[0].rij, nl->L[0].shift, nl->L[1].j, nl->L[1].owner, nl->L[1].rij, nl->L[1].shift);
    GNEP_CHECK_LAUNCH("k_compact");
  } else {
    k_pairs<<<blocks_for((int64_t)N * 32, 128), 128, 0, st>>>(
        N, nl->struct_off, nl->atom_struct, nl->pos, nl->cell, kr, tw, hsplit, frac, phi, plo, lp, off0, off1,
        nl->L[0].j, nl->L[0].owner, nl->L[0].rij, nl->L[0].shift, nl->L[1].j, nl->L[1].owner, nl->L[1].rij,
        nl->L[1].shift);
    GNEP_CHECK_LAUNCH("k_pairs<fill>");
  }
  {  // reverse entries of the angular list (the radial force terms need none)
    PairList& P = nl->L[1];
    if (P.n > 0)
      k_reverse<<<blocks_for(P.n, 256), 256, 0, st>>>(P.n, P.off, P.j, P.owner, P.shift, P.rev, m->err);
  }
  GNEP_CHECK_LAUNCH("k_reverse");
  cleanup();  // the reverse search sets kErrRevMissing, read at the end of the build
  return GNEP_OK;
}

}  // namespace gnep
