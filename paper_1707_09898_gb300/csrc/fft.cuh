// Shared-memory batched FFT engine for the stray-field convolution (sm_103a).
//
// The convolution of Sec. "Discretization" (Eq. (convolution)) is evaluated in
// Fourier space; only the product N^(k) M^(k) needs the frequency index, so the
// forward transforms are in-place mixed-radix decimation-in-frequency (natural
// order in, digit-reversed order out) and the inverse transforms are the exact
// reverse decimation-in-time (digit-reversed in, natural out). No reordering
// pass is ever made.
//
// A tile holds 16 lines of one length-L transform in shared memory, element
// (pos, line) in row pos at column line ^ swz(pos), swz(pos) = (pos ^ pos>>4) & 15.
// A half-warp covering the 16 lines of one position touches one 128-byte row
// (bank-conflict free for any radix pattern); the XOR swizzle also spreads a
// half-warp covering 16 positions of one line (the x passes read and write rows
// of the grid that way) over distinct banks. Radices are 32, 16, 8, 4, 2 and 3
// (in-register DFTs); lengths are L = 2^a 3^b with b <= 2, 8 <= L <= 1024.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tmk {

constexpr int TB = 16;  // lines per tile

// tile index of (pos, line); SW selects the XOR-swizzled layout (x passes)
template <bool SW>
__device__ __forceinline__ int tidx(int pos, int line) {
  if (SW) return pos * TB + (line ^ ((pos ^ (pos >> 4)) & 15));
  return pos * TB + line;
}
__device__ __forceinline__ int tix(int pos, int line) { return tidx<true>(pos, line); }

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return mk(a.x * s, a.y * s); }
// a * w
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> w) {
  return mk(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// a * conj(w)
template <typename T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> w) {
  return mk(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
template <typename T>
__device__ __forceinline__ cx<T> zero() { return mk<T>(T(0), T(0)); }

// ---------------------------------------------------------------------------
// Exact values cos(2 pi m / 32), m = 0..8 (the rest follow by symmetry).
__host__ __device__ constexpr double cos32_q(int m) {
  return m == 0 ? 1.0
       : m == 1 ? 0.980785280403230449126
       : m == 2 ? 0.923879532511286756128
       : m == 3 ? 0.831469612302545237079
       : m == 4 ? 0.707106781186547524401
       : m == 5 ? 0.555570233019602224743
       : m == 6 ? 0.382683432365089771728
       : m == 7 ? 0.195090322016128267848
                : 0.0;
}
// cos and sin of 2 pi m / 32 for m in [0, 16)
__host__ __device__ constexpr double cos32(int m) { return m <= 8 ? cos32_q(m) : -cos32_q(16 - m); }
__host__ __device__ constexpr double sin32(int m) { return m <= 8 ? cos32_q(8 - m) : cos32_q(m - 8); }
constexpr double kSqrt3Half = 0.866025403784438646764;

// a * W_32^m with W = exp(-2 pi i / 32) (forward) or its conjugate (inverse); m in [0,16)
template <typename T, bool INV>
__device__ __forceinline__ cx<T> tw32(cx<T> a, int m) {
  if (m == 0) return a;
  if (m == 8) return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
  const T c = T(cos32(m)), s = T(sin32(m));
  if (!INV) return mk(a.x * c + a.y * s, a.y * c - a.x * s);
  return mk(a.x * c - a.y * s, a.y * c + a.x * s);
}

// In-register DFT of size N (natural order in and out). Forward uses
// exp(-2 pi i jk / N), inverse exp(+2 pi i jk / N), both unnormalised.
template <typename T, int N, bool INV>
struct Dft {
  static __device__ __forceinline__ void run(cx<T>* v) {
    static_assert(N == 2 || N == 4 || N == 8 || N == 16 || N == 32, "radix");
    cx<T> e[N / 2], o[N / 2];
#pragma unroll
    for (int i = 0; i < N / 2; i++) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    Dft<T, N / 2, INV>::run(e);
    Dft<T, N / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < N / 2; k++) {
      cx<T> t = tw32<T, INV>(o[k], k * (32 / N));
      v[k] = e[k] + t;
      v[k + N / 2] = e[k] - t;
    }
  }
};
template <typename T, bool INV>
struct Dft<T, 1, INV> {
  static __device__ __forceinline__ void run(cx<T>*) {}
};
template <typename T, bool INV>
struct Dft<T, 3, INV> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> t = v[1] + v[2], d = v[1] - v[2];
    cx<T> m = v[0] - scale(t, T(0.5));
    cx<T> s = scale(d, T(kSqrt3Half));
    v[0] = v[0] + t;
    if (!INV) {
      v[1] = mk(m.x + s.y, m.y - s.x);
      v[2] = mk(m.x - s.y, m.y + s.x);
    } else {
      v[1] = mk(m.x - s.y, m.y + s.x);
      v[2] = mk(m.x + s.y, m.y - s.x);
    }
  }
};

// ---------------------------------------------------------------------------
// The radix-2 DFTs again (float only), with every butterfly whose twiddle is not 1 or
// -+i in fused multiply-adds: lo = a + W b in four FMAs and hi = a - W b as 2 a - lo in
// two, six instructions where the plain form takes eight (four for W b, four for the
// sum and difference). hi then carries the rounding error of lo with the opposite sign,
// a few float32 ulps more per transform. The compute-bound fused y/z kernels use them.
template <bool INV>
__device__ __forceinline__ void bfly_tw(cx<float>& lo, cx<float>& hi, cx<float> a, cx<float> b, int m) {
  // W = exp(-2 pi i / 32) forward, exp(+2 pi i / 32) inverse; m in [0, 16)
  if (m == 0) {
    lo = a + b;
    hi = a - b;
    return;
  }
  if (m == 8) {
    const cx<float> t = INV ? mk(-b.y, b.x) : mk(b.y, -b.x);
    lo = a + t;
    hi = a - t;
    return;
  }
  const float c = float(cos32(m)), s = INV ? -float(sin32(m)) : float(sin32(m));
  lo.x = __fmaf_rn(b.y, s, __fmaf_rn(b.x, c, a.x));   // a.x + (W b).x
  lo.y = __fmaf_rn(-b.x, s, __fmaf_rn(b.y, c, a.y));  // a.y + (W b).y
  hi.x = __fmaf_rn(2.0f, a.x, -lo.x);
  hi.y = __fmaf_rn(2.0f, a.y, -lo.y);
}
// a + W^m b only (the lower half of a butterfly)
template <bool INV>
__device__ __forceinline__ cx<float> bfly_lo(cx<float> a, cx<float> b, int m) {
  if (m == 0) return a + b;
  if (m == 8) return a + (INV ? mk(-b.y, b.x) : mk(b.y, -b.x));
  const float c = float(cos32(m)), s = INV ? -float(sin32(m)) : float(sin32(m));
  return mk(__fmaf_rn(b.y, s, __fmaf_rn(b.x, c, a.x)), __fmaf_rn(-b.x, s, __fmaf_rn(b.y, c, a.y)));
}

template <int N, bool INV>
struct DftF {
  static __device__ __forceinline__ void run(cx<float>* v) {
    static_assert(N == 2 || N == 4 || N == 8 || N == 16 || N == 32, "radix");
    cx<float> e[N / 2], o[N / 2];
#pragma unroll
    for (int i = 0; i < N / 2; i++) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    DftF<N / 2, INV>::run(e);
    DftF<N / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < N / 2; k++) bfly_tw<INV>(v[k], v[k + N / 2], e[k], o[k], k * (32 / N));
  }
};
template <bool INV>
struct DftF<1, INV> {
  static __device__ __forceinline__ void run(cx<float>*) {}
};

// Outputs 0 .. N/2 - 1 only (an inverse transform whose upper half is cropped).
template <int N, bool INV>
__device__ __forceinline__ void dft_low_half(cx<float>* v) {
  cx<float> e[N / 2], o[N / 2];
#pragma unroll
  for (int i = 0; i < N / 2; i++) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  DftF<N / 2, INV>::run(e);
  DftF<N / 2, INV>::run(o);
#pragma unroll
  for (int k = 0; k < N / 2; k++) v[k] = bfly_lo<INV>(e[k], o[k], k * (32 / N));
}

// 32-point DFT of inputs 0 .. 15 (inputs 16 .. 31 zero, a zero-padded transform):
// X[2m] = DFT16(x)[m] and X[2m+1] = DFT16(x[n] W32^n)[m]. v[0..15] in, v[0..31] out.
template <bool INV>
__device__ __forceinline__ void dft32_half_input(cx<float>* v) {
  cx<float> a[16], b[16];
#pragma unroll
  for (int n = 0; n < 16; n++) {
    a[n] = v[n];
    b[n] = tw32<float, INV>(v[n], n);
  }
  DftF<16, INV>::run(a);
  DftF<16, INV>::run(b);
#pragma unroll
  for (int m = 0; m < 16; m++) {
    v[2 * m] = a[m];
    v[2 * m + 1] = b[m];
  }
}

// ---------------------------------------------------------------------------
// Plans: L = 2^a 3^b. The power-of-two part is one stage (when b > 0 and
// a <= 5) or two near-equal stages; then b radix-3 stages. Every plan has at
// least two stages.
__host__ __device__ constexpr int exp2_of(int L) {
  int a = 0;
  while (L > 1 && L % 2 == 0) { L /= 2; a++; }
  return a;
}
__host__ __device__ constexpr int exp3_of(int L) {
  int b = 0;
  while (L > 1 && L % 3 == 0) { L /= 3; b++; }
  return b;
}
__host__ __device__ constexpr bool two_pow2_stages(int L) { return exp3_of(L) == 0 || exp2_of(L) > 5; }
__host__ __device__ constexpr int plan_stages(int L) {
  return (two_pow2_stages(L) ? 2 : (exp2_of(L) > 0 ? 1 : 0)) + exp3_of(L);
}
__host__ __device__ constexpr int plan_radix(int L, int s) {
  if (two_pow2_stages(L)) {
    const int a = exp2_of(L), a1 = (a + 1) / 2, a2 = a - a1;
    if (s == 0) return 1 << a1;
    if (s == 1) return 1 << a2;
    return 3;
  }
  if (s == 0) return 1 << exp2_of(L);
  return 3;
}
// G_s = L / (R_0 ... R_{s-1}): size of the sub-transforms stage s works on
__host__ __device__ constexpr int plan_span(int L, int s) {
  int G = L;
  for (int t = 0; t < s; t++) G /= plan_radix(L, t);
  return G;
}
__host__ __device__ constexpr bool supported_length(int L) {
  if (L < 8 || L > 1024 || L % 2 != 0) return false;
  int r = L;
  while (r % 2 == 0) r /= 2;
  while (r % 3 == 0) r /= 3;
  return r == 1 && exp3_of(L) <= 2;
}

// Position (after the forward DIF) of frequency k, and its inverse.
template <int L>
__device__ __forceinline__ int pos_of_k(int k) {
  int pos = 0, span = L, rem = k;
#pragma unroll
  for (int s = 0; s < plan_stages(L); s++) {
    const int R = plan_radix(L, s);
    span /= R;
    pos += (rem % R) * span;
    rem /= R;
  }
  return pos;
}
template <int L>
__device__ __forceinline__ int k_of_pos(int pos) {
  constexpr int S = plan_stages(L);
  int d[S > 0 ? S : 1];
  int rem = pos;
#pragma unroll
  for (int s = S - 1; s >= 0; s--) {
    const int R = plan_radix(L, s);
    d[s] = rem % R;
    rem /= R;
  }
  int k = 0, m = 1;
#pragma unroll
  for (int s = 0; s < S; s++) {
    k += d[s] * m;
    m *= plan_radix(L, s);
  }
  return k;
}

// ---------------------------------------------------------------------------
// Stage kernels on a tile. Unit u of stage s: line = u % 16, t = u / 16,
// group g = t / M, j = t % M; it owns positions g*G + j + q*M, q < R.
template <int L, int s>
struct StageShape {
  static constexpr int R = plan_radix(L, s);
  static constexpr int G = plan_span(L, s);
  static constexpr int M = G / R;
  static constexpr int NU = (L / R) * TB;  // units per stage
};

// twiddle for DIF output q / DIT input q of unit (j): W_G^{jq} = tw[j q L/G]
template <typename T, int L, int s, bool INV>
__device__ __forceinline__ void apply_twiddles(cx<T>* v, int j, const cx<T>* tw) {
  using S = StageShape<L, s>;
  if (S::M == 1) return;
  if (j == 0) return;
#pragma unroll
  for (int q = 1; q < S::R; q++) {
    const cx<T> w = tw[(j * q) * (L / S::G)];
    v[q] = INV ? cmulc(v[q], w) : cmul(v[q], w);
  }
}

// Tile index of position base + q M of a stage unit. For a radix-16 unit with M = 1 in
// the swizzled layout the positions are g 16 + q, whose swizzle is q ^ (g mod 16): one
// XOR per element instead of the general shift-and-mask.
template <int R, int M, bool SW>
__device__ __forceinline__ int unit_idx(int g, int base, int q, int line) {
  if constexpr (SW && R == TB && M == 1) return g * (TB * TB) + q * TB + ((line ^ (g & 15)) ^ q);
  else return tidx<SW>(base + q * M, line);
}

// One forward DIF stage in place on the tile.
template <typename T, int L, int s, int NT, bool SW = false>
__device__ __forceinline__ void dif_stage(cx<T>* tile, const cx<T>* tw) {
  using S = StageShape<L, s>;
  constexpr int ITER = (S::NU + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, t = u / TB, g = t / S::M, j = t % S::M;
      const int base = g * S::G + j;
      cx<T> v[S::R];
#pragma unroll
      for (int q = 0; q < S::R; q++) v[q] = tile[unit_idx<S::R, S::M, SW>(g, base, q, line)];
      Dft<T, S::R, false>::run(v);
      apply_twiddles<T, L, s, false>(v, j, tw);
#pragma unroll
      for (int q = 0; q < S::R; q++) tile[unit_idx<S::R, S::M, SW>(g, base, q, line)] = v[q];
    }
  }
}

// One inverse DIT stage in place on the tile.
template <typename T, int L, int s, int NT, bool SW = false>
__device__ __forceinline__ void dit_stage(cx<T>* tile, const cx<T>* tw) {
  using S = StageShape<L, s>;
  constexpr int ITER = (S::NU + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, t = u / TB, g = t / S::M, j = t % S::M;
      const int base = g * S::G + j;
      cx<T> v[S::R];
#pragma unroll
      for (int q = 0; q < S::R; q++) v[q] = tile[unit_idx<S::R, S::M, SW>(g, base, q, line)];
      apply_twiddles<T, L, s, true>(v, j, tw);
      Dft<T, S::R, true>::run(v);
#pragma unroll
      for (int q = 0; q < S::R; q++) tile[unit_idx<S::R, S::M, SW>(g, base, q, line)] = v[q];
    }
  }
}

// Stage 0 forward, reading its inputs through ld(pos, line) (zero beyond the
// valid range is the loader's job) and writing the tile. All loads of a thread
// are issued before any arithmetic.
template <typename T, int L, int NT, typename LD, bool SW = false>
__device__ __forceinline__ void dif_stage0_load(cx<T>* tile, const cx<T>* tw, LD ld) {
  using S = StageShape<L, 0>;
  constexpr int ITER = (S::NU + NT - 1) / NT;
  cx<T> v[ITER][S::R];
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, j = u / TB;
#pragma unroll
      for (int q = 0; q < S::R; q++) v[it][q] = ld(j + q * S::M, line);
    }
  }
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, j = u / TB;
      Dft<T, S::R, false>::run(v[it]);
      apply_twiddles<T, L, 0, false>(v[it], j, tw);
#pragma unroll
      for (int q = 0; q < S::R; q++) tile[tidx<SW>(j + q * S::M, line)] = v[it][q];
    }
  }
}

// Last forward stage (M = 1), writing its outputs through st(pos, line, v).
template <typename T, int L, int NT, typename ST, bool SW = false>
__device__ __forceinline__ void dif_last_store(const cx<T>* tile, ST st) {
  constexpr int s = plan_stages(L) - 1;
  using S = StageShape<L, s>;
  static_assert(S::M == 1, "last stage");
  constexpr int ITER = (S::NU + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, g = u / TB;
      cx<T> v[S::R];
#pragma unroll
      for (int q = 0; q < S::R; q++) v[q] = tile[tidx<SW>(g * S::R + q, line)];
      Dft<T, S::R, false>::run(v);
#pragma unroll
      for (int q = 0; q < S::R; q++) st(g * S::R + q, line, v[q]);
    }
  }
}

// First inverse stage (the last plan stage, M = 1) reading ld(pos, line).
template <typename T, int L, int NT, typename LD, bool SW = false>
__device__ __forceinline__ void dit_last_load(cx<T>* tile, LD ld) {
  constexpr int s = plan_stages(L) - 1;
  using S = StageShape<L, s>;
  static_assert(S::M == 1, "last stage");
  constexpr int ITER = (S::NU + NT - 1) / NT;
  cx<T> v[ITER][S::R];
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, g = u / TB;
#pragma unroll
      for (int q = 0; q < S::R; q++) v[it][q] = ld(g * S::R + q, line);
    }
  }
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, g = u / TB;
      Dft<T, S::R, true>::run(v[it]);
#pragma unroll
      for (int q = 0; q < S::R; q++) tile[tidx<SW>(g * S::R + q, line)] = v[it][q];
    }
  }
}

// Last inverse stage (plan stage 0), natural-order outputs through st(pos, line, v).
template <typename T, int L, int NT, typename ST, bool SW = false>
__device__ __forceinline__ void dit_stage0_store(const cx<T>* tile, const cx<T>* tw, ST st) {
  using S = StageShape<L, 0>;
  constexpr int ITER = (S::NU + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * NT + threadIdx.x;
    if (S::NU % NT == 0 || u < S::NU) {
      const int line = u % TB, j = u / TB;
      cx<T> v[S::R];
#pragma unroll
      for (int q = 0; q < S::R; q++) v[q] = tile[tidx<SW>(j + q * S::M, line)];
      apply_twiddles<T, L, 0, true>(v, j, tw);
      Dft<T, S::R, true>::run(v);
#pragma unroll
      for (int q = 0; q < S::R; q++) st(j + q * S::M, line, v[q]);
    }
  }
}

// Helpers running stage ranges with a block barrier after each stage.
template <typename T, int L, int NT, int s, int e, bool SW = false>
struct DifRange {
  static __device__ __forceinline__ void run(cx<T>* tile, const cx<T>* tw) {
    if constexpr (s < e) {
      dif_stage<T, L, s, NT, SW>(tile, tw);
      __syncthreads();
      DifRange<T, L, NT, s + 1, e, SW>::run(tile, tw);
    }
  }
};
// inverse stages s = hi-1 down to lo
template <typename T, int L, int NT, int lo, int hi, bool SW = false>
struct DitRange {
  static __device__ __forceinline__ void run(cx<T>* tile, const cx<T>* tw) {
    if constexpr (hi > lo) {
      dit_stage<T, L, hi - 1, NT, SW>(tile, tw);
      __syncthreads();
      DitRange<T, L, NT, lo, hi - 1, SW>::run(tile, tw);
    }
  }
};

// frequency of the R consecutive positions g*R + q of the last stage (radix R):
// k = k_of_pos(g*R) + q * (L / R)
template <int L>
__device__ __forceinline__ int k_of_group(int g) {
  constexpr int S = plan_stages(L);
  return k_of_pos<L>(g * plan_radix(L, S - 1));
}

// Cooperative copy of the length-L twiddle table W_L^m into shared memory.
template <typename T, int NT>
__device__ __forceinline__ void load_twiddles(cx<T>* dst, const cx<T>* src, int L) {
  for (int i = threadIdx.x; i < L; i += NT) dst[i] = src[i];
}

}  // namespace tmk
