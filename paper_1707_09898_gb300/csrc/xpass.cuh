// Pieces shared by the x-axis passes of the stray-field convolution (k_xfwd.cu,
// k_xinv.cu; Sec. "Discretization", Eq. (convolution)).
//
// A block works on 32 real rows: rows 2 l and 2 l + 1 travel as line l of a 16-line
// tile (row a + i row b), transformed together and separated into their half spectra
// kx = 0..L/2 afterwards; the inverse extends the half spectra by Hermitian symmetry.
// The tile uses the swizzled layout of fft.cuh so that both the x-fastest global
// accesses and the line-fastest FFT stages are free of bank conflicts.
//
// For L = 2 kNT (L = 512, the 256-cell grids) every thread owns one frequency
// k < L/2 of the half spectra: the tile positions of k and L - k and their swizzles
// are computed once per thread, the 16 lines are unrolled, and the global rows are
// read and written with consecutive threads on consecutive k. Other lengths take the
// general loops below.
#pragma once
#include "fft.cuh"
#include "internal.h"

namespace tmk {

namespace {

constexpr int ROWS = 2 * TB;  // real rows per block

template <int L>
__host__ __device__ constexpr bool k_per_thread() {
  return L / 2 == kNT;
}

__device__ __forceinline__ int swz(int pos) { return (pos ^ (pos >> 4)) & 15; }

// tile index of x = j + q M of a stage-0 unit; when M == TB (j < 16) the swizzle of
// that position is j ^ (q mod 16)
template <int M>
__device__ __forceinline__ int tix0(int j, int q, int line) {
  if constexpr (M == TB) return (j + q * TB) * TB + ((line ^ j) ^ (q & 15));
  else return tix(j + q * M, line);
}

__device__ __forceinline__ float ipow(float r, float p) {
  if (p == 3.0f) return r * r * r;
  if (p == 2.0f) return r * r;
  if (p == 1.0f) return r;
  return powf(r, p);
}
__device__ __forceinline__ float dpow(float r, float p) {  // p r^(p-1)
  if (p == 3.0f) return 3.0f * r * r;
  if (p == 2.0f) return 2.0f * r;
  if (p == 1.0f) return 1.0f;
  return p * powf(r, p - 1.0f);
}
// the same with p = 3 fixed at compile time (the paper's penalisation exponent)
template <bool P3>
__device__ __forceinline__ float ipow_t(float r, float p) {
  if constexpr (P3) return r * r * r;
  else return ipow(r, p);
}
template <bool P3>
__device__ __forceinline__ float dpow_t(float r, float p) {
  if constexpr (P3) return 3.0f * r * r;
  else return dpow(r, p);
}

// Stage-0 twiddles W_L^(j q) laid out [q][j] (j fastest), so that the 16 threads of a
// half-warp, which hold consecutive j of one q, read consecutive words.
template <int L>
__device__ __forceinline__ void load_twiddles0(cx<float>* tw0, const cx<float>* tw) {
  constexpr int M = StageShape<L, 0>::M;
  for (int i = threadIdx.x; i < L; i += kNT) {
    const int q = i / M, j = i - q * M;
    tw0[i] = tw[j * q];  // j q <= (M - 1)(R - 1) < L
  }
}
template <int L, bool INV>
__device__ __forceinline__ void twiddle0(cx<float>* v, int j, const cx<float>* tw0) {
  using S0 = StageShape<L, 0>;
  if (j == 0) return;
#pragma unroll
  for (int q = 1; q < S0::R; q++) {
    const cx<float> w = tw0[q * S0::M + j];
    v[q] = INV ? cmulc(v[q], w) : cmul(v[q], w);
  }
}

// Last inverse stage (plan stage 0) with x fastest; fn(it, j, line, v[R]) receives the
// natural-order outputs at x = j + q M and may write new stage-0 inputs back into v
// and return true, in which case the forward stage 0 is applied to v in place.
template <int L, typename FN>
__device__ __forceinline__ void xdit0(cx<float>* tile, const cx<float>* tw0, FN fn) {
  using S0 = StageShape<L, 0>;
  constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * kNT + threadIdx.x;
    if (NU % kNT == 0 || u < NU) {
      const int j = u % M, line = u / M;
      cx<float> v[R];
#pragma unroll
      for (int q = 0; q < R; q++) v[q] = tile[tix0<M>(j, q, line)];
      twiddle0<L, true>(v, j, tw0);
      Dft<float, R, true>::run(v);
      if (fn(it, j, line, v)) {
        Dft<float, R, false>::run(v);
        twiddle0<L, false>(v, j, tw0);
#pragma unroll
        for (int q = 0; q < R; q++) tile[tix0<M>(j, q, line)] = v[q];
      }
    }
  }
}

// Half spectra of the 2*TB rows from the finished forward transform into
// out[row][k] (rows row0.., k < P; zero for L/2 < k < P).
template <int L>
__device__ __forceinline__ void xseparate(const cx<float>* tile, cx<float>* out, int row0, int rows, int P) {
  if constexpr (k_per_thread<L>()) {
    const int k = threadIdx.x, nr = rows - row0;
    const int pa = pos_of_k<L>(k), pb = pos_of_k<L>((L - k) % L);
    const cx<float>* ta = tile + pa * TB;
    const cx<float>* tb = tile + pb * TB;
    const int ca = swz(pa), cb = swz(pb);
    cx<float>* dst = out + (long long)row0 * P + k;
#pragma unroll
    for (int l = 0; l < TB; l++) {
      const cx<float> Z = ta[l ^ ca], Zm = tb[l ^ cb];
      if (2 * l < nr) dst[(2 * l) * P] = mk(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));       // (Z + conj Zm) / 2
      if (2 * l + 1 < nr) dst[(2 * l + 1) * P] = mk(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));  // (Z - conj Zm) / 2i
    }
    // k = L/2 (A = Re Z, B = Im Z) and the zero columns up to P, 16 columns of a row at a time
    const int W = P - L / 2;
    const int pn = pos_of_k<L>(L / 2);
    for (int rr = threadIdx.x / 16; rr < 2 * TB && rr < nr; rr += kNT / 16) {
      for (int c = threadIdx.x % 16; c < W; c += 16) {
        cx<float> v = zero<float>();
        if (c == 0) {
          const cx<float> Z = tile[tix(pn, rr >> 1)];
          v = (rr & 1) ? mk(Z.y, 0.0f) : mk(Z.x, 0.0f);
        }
        out[(long long)(row0 + rr) * P + L / 2 + c] = v;
      }
    }
  } else {
    for (int i = threadIdx.x; i < TB * P; i += kNT) {
      const int line = i / P, k = i - line * P;
      cx<float> A = zero<float>(), B = zero<float>();
      if (k <= L / 2) {
        const cx<float> Z = tile[tix(pos_of_k<L>(k), line)];
        const cx<float> Zm = tile[tix(pos_of_k<L>((L - k) % L), line)];
        A = mk(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
        B = mk(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));
      }
      const int ra = row0 + 2 * line;
      if (ra < rows) out[(long long)ra * P + k] = A;
      if (ra + 1 < rows) out[(long long)(ra + 1) * P + k] = B;
    }
  }
}

// Hermitian extension of the half spectra of 2*TB rows into the tile (DIF positions).
// Every global load of the block is issued before the first shared store.
template <int L>
__device__ __forceinline__ void xhermitian(cx<float>* tile, const cx<float>* in, int row0, int rows, int P) {
  if constexpr (k_per_thread<L>()) {
    const int k = threadIdx.x, nr = rows - row0;
    const cx<float>* src = in + (long long)row0 * P + k;
    cx<float> A[TB], B[TB];
#pragma unroll
    for (int l = 0; l < TB; l++) {
      A[l] = 2 * l < nr ? src[(2 * l) * P] : zero<float>();
      B[l] = 2 * l + 1 < nr ? src[(2 * l + 1) * P] : zero<float>();
    }
    cx<float> An = zero<float>(), Bn = zero<float>();  // k = L/2 of line threadIdx.x
    if (threadIdx.x < TB) {
      const int l = threadIdx.x;
      const cx<float>* s = in + (long long)row0 * P + L / 2;
      if (2 * l < nr) An = s[(2 * l) * P];
      if (2 * l + 1 < nr) Bn = s[(2 * l + 1) * P];
    }
    const int pa = pos_of_k<L>(k), pb = pos_of_k<L>((L - k) % L);
    cx<float>* ta = tile + pa * TB;
    cx<float>* tb = tile + pb * TB;
    const int ca = swz(pa), cb = swz(pb);
    if (k == 0) {
#pragma unroll
      for (int l = 0; l < TB; l++) ta[l ^ ca] = mk(A[l].x, B[l].x);
    } else {
#pragma unroll
      for (int l = 0; l < TB; l++) {
        const cx<float> a = A[l], b = B[l];
        ta[l ^ ca] = mk(a.x - b.y, a.y + b.x);  // A + iB
        tb[l ^ cb] = mk(a.x + b.y, b.x - a.y);  // conj(A) + i conj(B)
      }
    }
    if (threadIdx.x < TB) tile[tix(pos_of_k<L>(L / 2), threadIdx.x)] = mk(An.x, Bn.x);
  } else {
    constexpr int K = L / 2 + 1;
    constexpr int N = TB * K, ITER = (N + kNT - 1) / kNT;
    cx<float> A[ITER], B[ITER];
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int i = it * kNT + threadIdx.x;
      const int line = i / K, k = i - line * K;
      const int ra = row0 + 2 * line, rb = ra + 1;
      const bool ok = N % kNT == 0 || i < N;
      A[it] = (ok && ra < rows) ? in[(long long)ra * P + k] : zero<float>();
      B[it] = (ok && rb < rows) ? in[(long long)rb * P + k] : zero<float>();
    }
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int i = it * kNT + threadIdx.x;
      if (N % kNT != 0 && i >= N) continue;
      const int line = i / K, k = i - line * K;
      const cx<float> a = A[it], b = B[it];
      if (k == 0 || k == L / 2) {
        tile[tix(pos_of_k<L>(k), line)] = mk(a.x, b.x);
      } else {
        tile[tix(pos_of_k<L>(k), line)] = mk(a.x - b.y, a.y + b.x);      // A + iB
        tile[tix(pos_of_k<L>(L - k), line)] = mk(a.x + b.y, b.x - a.y);  // conj(A) + i conj(B)
      }
    }
  }
}

// shared memory of an x-pass block: twiddles, stage-0 twiddles, tile
template <int L>
size_t xsmem() {
  return (size_t)(2 * L + L * TB) * sizeof(float2);
}

}  // namespace

}  // namespace tmk
