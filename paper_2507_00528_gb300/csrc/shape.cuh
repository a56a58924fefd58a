// Compile-time model shape of the sweeps: species, radial and angular channels
// and basis sizes, the 4-body term and the angular degree l_max.
#pragma once

namespace gnep {

template <int NS_, int NQR_, int KR_, int NQA_, int KA_, bool FB_, int LMAX_ = 4>
struct Sh {
  static constexpr int NS = NS_, NQR = NQR_, KR = KR_, NQA = NQA_, KA = KA_, LMAX = LMAX_;
  static constexpr bool FB = FB_;
  static constexpr int NLX = (LMAX + 1) * (LMAX + 1) - 1;  // (l, m) components for l = 1..l_max
  static constexpr int NDES = NQR + NQA * LMAX + (FB ? NQA : 0);
  __host__ __device__ static constexpr int vang(int n, int l) { return NQR + n * LMAX + (l - 1); }
  __host__ __device__ static constexpr int v4b(int n) { return NQR + NQA * LMAX + n; }
  static constexpr int NCR = NS * NS * NQR * KR;
  static constexpr int NCA = NS * NS * NQA * KA;
  static constexpr int NQ = NQR > NQA ? NQR : NQA;
};

}  // namespace gnep
