// x-axis passes of the stray-field convolution (Sec. "Discretization", Eq. (convolution)).
//
// Forward: real rows (rho^p, rho^p M0_c of Sec. "Methodology" Eq. 2, or a given
// vector component) are zero padded from nx to L (the first DIF stage reads only
// x < nx) and transformed two rows at a time (row a + i row b), then separated
// into the half spectra kx = 0..L/2. One block per (32-row tile, component).
// Inverse: half spectra are extended by Hermitian symmetry, two rows are
// recovered from one complex inverse transform, cropped to nx, and handed to a
// sink: write H; the least-squares objective and dJ/dH, whose zero-padded
// forward x transform (the adjoint source) starts in the same registers; or the
// chain rule dJ/drho = p rho^(p-1) M0 . (D g) (Sec. "Methodology",
// Eqs. (adjoint1)-(adjoint2)).
// The first forward and the last inverse stage map consecutive threads to
// consecutive x of one row pair, so global rows are read and written in
// 64-byte runs straight from registers; the half-spectrum rows are read and
// written with consecutive threads on consecutive kx. The swizzled tile keeps
// both orientations free of bank conflicts, and no staging buffer is needed.
#include "fft.cuh"
#include "internal.h"

namespace tmk {

namespace {

constexpr int ROWS = 2 * TB;  // real rows per block

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

// Units of plan stage 0 with x fastest: unit u -> (j = u % M, line = u / M),
// positions j + q M (q < R). Forward reads go through ld(x, line).
template <int L, typename LD>
__device__ __forceinline__ void xdif0(cx<float>* tile, const cx<float>* tw, LD ld) {
  using S0 = StageShape<L, 0>;
  constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
  cx<float> v[ITER][R];
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * kNT + threadIdx.x;
    if (NU % kNT == 0 || u < NU) {
      const int j = u % M, line = u / M;
#pragma unroll
      for (int q = 0; q < R; q++) v[it][q] = ld(j + q * M, line);
    }
  }
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * kNT + threadIdx.x;
    if (NU % kNT == 0 || u < NU) {
      const int j = u % M, line = u / M;
      Dft<float, R, false>::run(v[it]);
      apply_twiddles<float, L, 0, false>(v[it], j, tw);
#pragma unroll
      for (int q = 0; q < R; q++) tile[tix(j + q * M, line)] = v[it][q];
    }
  }
}

// Last inverse stage (plan stage 0) with x fastest; fn(it, j, line, v[R]) receives the
// natural-order outputs at x = j + q M and may write new stage-0 inputs back into v
// and return true, in which case the forward stage 0 is applied to v in place.
template <int L, typename FN>
__device__ __forceinline__ void xdit0(cx<float>* tile, const cx<float>* tw, FN fn) {
  using S0 = StageShape<L, 0>;
  constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * kNT + threadIdx.x;
    if (NU % kNT == 0 || u < NU) {
      const int j = u % M, line = u / M;
      cx<float> v[R];
#pragma unroll
      for (int q = 0; q < R; q++) v[q] = tile[tix(j + q * M, line)];
      apply_twiddles<float, L, 0, true>(v, j, tw);
      Dft<float, R, true>::run(v);
      if (fn(it, j, line, v)) {
        Dft<float, R, false>::run(v);
        apply_twiddles<float, L, 0, false>(v, j, tw);
#pragma unroll
        for (int q = 0; q < R; q++) tile[tix(j + q * M, line)] = v[q];
      }
    }
  }
}

// Half spectra of the 2*TB rows from the finished forward transform: kx fastest.
template <int L, typename OUT>
__device__ __forceinline__ void xseparate(const cx<float>* tile, int P, OUT out) {
  for (int i = threadIdx.x; i < TB * P; i += kNT) {
    const int line = i / P, k = i - line * P;
    cx<float> A = zero<float>(), B = zero<float>();
    if (k <= L / 2) {
      const cx<float> Z = tile[tix(pos_of_k<L>(k), line)];
      const cx<float> Zm = tile[tix(pos_of_k<L>((L - k) % L), line)];
      A = mk(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));  // (Z + conj Zm) / 2
      B = mk(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));  // (Z - conj Zm) / 2i
    }
    out(2 * line, k, A);
    out(2 * line + 1, k, B);
  }
}

// Hermitian extension of the half spectra of 2*TB rows into the tile (DIF positions).
// Every global load of the block is issued before the first shared store.
template <int L>
__device__ __forceinline__ void xhermitian(cx<float>* tile, const cx<float>* in, int row0, int rows, int P) {
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

// Persistent forward x pass: a block loops over 32-row tiles; the raw inputs of
// the next tile are loaded into registers while the current tile is separated
// and stored, so global latency overlaps the shared-memory work.
template <int L, int SRC>
__global__ void __launch_bounds__(kNT, 2) k_xfwd(XFwdArgs a) {
  constexpr int S = plan_stages(L);
  using S0 = StageShape<L, 0>;
  constexpr bool withM0 = SRC == SRC_RHO_M0;
  constexpr int RM = withM0 ? 1 : 0;
  constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
  // nx <= L/2, so the stage-0 inputs x = j + q M with q >= R/2 are always padding
  constexpr int RH = R / 2 > 0 ? R / 2 : 1;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int c = a.comp[blockIdx.y];
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[blockIdx.y] * a.out_cstride;
  const int ntiles = (a.rows + ROWS - 1) / ROWS;
  const float* src = SRC == SRC_VECTOR ? a.vec + c * a.vec_cstride : a.rho;
  const float* m0 = withM0 ? a.M0v + c * a.M0v_cstride : nullptr;
  float ra[ITER][RH], rb[ITER][RH], ma[ITER][RM ? RH : 1], mb[ITER][RM ? RH : 1];
  auto fetch = [&](int t) {
    const int row0 = t * ROWS;
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      const int j = u % M, line = u / M;
      const int ra_ = row0 + 2 * line, rb_ = ra_ + 1;
      const bool ok = NU % kNT == 0 || u < NU;
#pragma unroll
      for (int q = 0; q < RH; q++) {
        const int x = j + q * M;
        const long long oa = (long long)ra_ * a.nx + x;
        const bool in_x = ok && x < a.nx;
        ra[it][q] = (in_x && ra_ < a.rows) ? src[oa] : 0.0f;
        rb[it][q] = (in_x && rb_ < a.rows) ? src[oa + a.nx] : 0.0f;
        if constexpr (withM0) {
          ma[it][q] = (in_x && ra_ < a.rows) ? m0[oa] : 0.0f;
          mb[it][q] = (in_x && rb_ < a.rows) ? m0[oa + a.nx] : 0.0f;
        }
      }
    }
  };
  int t = blockIdx.x;
  if (t < ntiles) fetch(t);
  __syncthreads();
  for (; t < ntiles; t += gridDim.x) {
    const int row0 = t * ROWS;
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (NU % kNT == 0 || u < NU) {
        const int j = u % M, line = u / M;
        cx<float> v[R];
#pragma unroll
        for (int q = RH; q < R; q++) v[q] = zero<float>();
#pragma unroll
        for (int q = 0; q < RH; q++) {
          float va = ra[it][q], vb = rb[it][q];
          if constexpr (SRC != SRC_VECTOR) {
            va = ipow(va, a.p);
            vb = ipow(vb, a.p);
            if constexpr (withM0) {
              va *= ma[it][q];
              vb *= mb[it][q];
            }
          }
          v[q] = mk(va, vb);
        }
        Dft<float, R, false>::run(v);
        apply_twiddles<float, L, 0, false>(v, j, tw);
#pragma unroll
        for (int q = 0; q < R; q++) tile[tix(j + q * M, line)] = v[q];
      }
    }
    __syncthreads();
    DifRange<float, L, kNT, 1, S, true>::run(tile, tw);
    if (t + (int)gridDim.x < ntiles) fetch(t + gridDim.x);
    xseparate<L>(tile, a.P, [&](int rr, int k, cx<float> v) {
      const int row = row0 + rr;
      if (row < a.rows) out[(long long)row * a.P + k] = v;
    });
    __syncthreads();
  }
}

// Called by every thread of every block after thread 0 wrote the block's J partial:
// the last block to finish sums the partials in index order (the order of a separate
// one-block reduction) into *Jout and re-arms the counter.
__device__ void finish_j(const XInvArgs& a) {
  __shared__ unsigned int last;
  __shared__ double r2[kNT];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(a.Jcount, 1u) == gridDim.x * gridDim.y - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int n = gridDim.x * gridDim.y;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kNT) s += __ldcg(a.Jpart + i);
  r2[threadIdx.x] = s;
  __syncthreads();
  for (int w = kNT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) r2[threadIdx.x] += r2[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *a.Jout = r2[0];
    *a.Jcount = 0u;
  }
}

template <int L, int SINK, int MINB>
__global__ void __launch_bounds__(kNT, MINB) k_xinv(XInvArgs a) {
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  __shared__ double red[kNT / 32];
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int row0 = a.row_base + blockIdx.x * ROWS;
  const cx<float>* in0 = reinterpret_cast<const cx<float>*>(a.in);

  if constexpr (SINK == SINK_CHAIN && MINB == 2) {
    // one slot, already contracted with the constant M0: G = p rho^(p-1) D
    using S0 = StageShape<L, 0>;
    constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
    constexpr int RH = R / 2 > 0 ? R / 2 : 1;  // x = j + q M < nx <= L/2 needs q < R/2
    __shared__ float wmax[kNT / 32];
    __syncthreads();
    xhermitian<L>(tile, in0 + a.in_slot[0] * a.in_cstride, row0, a.rows, a.P);
    // rho of this tile, fetched while the inverse stages run
    float pa[ITER][RH], pb[ITER][RH];
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      const int j = u % M, line = u / M;
      const int ra = row0 + 2 * line, rb = ra + 1;
      const bool ok = NU % kNT == 0 || u < NU;
#pragma unroll
      for (int q = 0; q < RH; q++) {
        const int x = j + q * M;
        const long long o = (long long)ra * a.nx + x;
        pa[it][q] = (ok && x < a.nx && ra < a.rows) ? a.rho[o] : 0.0f;
        pb[it][q] = (ok && x < a.nx && rb < a.rows) ? a.rho[o + a.nx] : 0.0f;
      }
    }
    __syncthreads();
    DitRange<float, L, kNT, 1, S, true>::run(tile, tw);
    float gm = 0.0f;
    xdit0<L>(tile, tw, [&](int it, int j, int line, cx<float>* v) {
      const int ra = row0 + 2 * line;
#pragma unroll
      for (int q = 0; q < RH; q++) {
        const int x = j + q * M;
        if (x >= a.nx) continue;
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int row = ra + h;
          if (row >= a.rows) continue;
          const long long o = (long long)row * a.nx + x;
          const float G = dpow(h ? pb[it][q] : pa[it][q], a.p) * (h ? v[q].y : v[q].x);
          a.G[o] = G;
          gm = fmaxf(gm, fabsf(G));
        }
      }
      return false;
    });
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kNT / 32; w++) gm = fmaxf(gm, wmax[w]);
      if (gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    }
    return;
  } else if constexpr (SINK == SINK_CHAIN) {
    using S0 = StageShape<L, 0>;
    constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
    float acc[ITER][R][2];
#pragma unroll
    for (int it = 0; it < ITER; it++)
#pragma unroll
      for (int q = 0; q < R; q++) acc[it][q][0] = acc[it][q][1] = 0.0f;
    for (int jc = 0; jc < a.ncomp; jc++) {
      __syncthreads();
      xhermitian<L>(tile, in0 + a.in_slot[jc] * a.in_cstride, row0, a.rows, a.P);
      __syncthreads();
      DitRange<float, L, kNT, 1, S, true>::run(tile, tw);
      const int c = a.comp[jc];
      xdit0<L>(tile, tw, [&](int it, int j, int line, cx<float>* v) {
        const int ra = row0 + 2 * line, rb = ra + 1;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int x = j + q * M;
          float ma = 1.0f, mb = 1.0f;  // contracted slot: coefficient 1
          if (a.M0v && x < a.nx) {
            if (ra < a.rows) ma = a.M0v[c * a.M0v_cstride + (long long)ra * a.nx + x];
            if (rb < a.rows) mb = a.M0v[c * a.M0v_cstride + (long long)rb * a.nx + x];
          }
          acc[it][q][0] += ma * v[q].x;
          acc[it][q][1] += mb * v[q].y;
        }
        return false;
      });
    }
    float gm = 0.0f;
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (NU % kNT == 0 || u < NU) {
        const int j = u % M, line = u / M;
        const int ra = row0 + 2 * line;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int x = j + q * M;
          if (x >= a.nx) continue;
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const int row = ra + h;
            if (row >= a.rows) continue;
            const long long o = (long long)row * a.nx + x;
            const float G = dpow(a.rho[o], a.p) * acc[it][q][h];
            a.G[o] = G;
            gm = fmaxf(gm, fabsf(G));
          }
        }
      }
    }
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((threadIdx.x & 31) == 0 && gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    return;
  } else {
  const int jc = blockIdx.y, c = a.comp[jc];
  const cx<float>* in = in0 + a.in_slot[jc] * a.in_cstride;
  if constexpr (SINK == SINK_OBJECTIVE) {
    if (a.ext) {  // only the rows of the target planes carry H (and the adjoint source)
      const long long lo = (long long)a.ext[0] * a.ny, hi = (long long)a.ext[1] * a.ny;
      if (row0 + ROWS <= lo || row0 >= hi) {
        if (threadIdx.x == 0) a.Jpart[jc * gridDim.x + blockIdx.x] = 0.0;
        if (a.Jcount) finish_j(a);
        return;
      }
    }
  }
  __syncthreads();
  xhermitian<L>(tile, in, row0, a.rows, a.P);
  __syncthreads();
  DitRange<float, L, kNT, 1, S, true>::run(tile, tw);

  if constexpr (SINK == SINK_FIELD) {
    xdit0<L>(tile, tw, [&](int, int j, int line, cx<float>* v) {
      const int ra = row0 + 2 * line, rb = ra + 1;
      constexpr int R = StageShape<L, 0>::R, M = StageShape<L, 0>::M;
#pragma unroll
      for (int q = 0; q < R; q++) {
        const int x = j + q * M;
        if (x >= a.nx) continue;
        if (ra < a.rows) a.H[c * a.H_cstride + (long long)ra * a.nx + x] = v[q].x;
        if (rb < a.rows) a.H[c * a.H_cstride + (long long)rb * a.nx + x] = v[q].y;
      }
      return false;
    });
    return;
  } else {
  // SINK_OBJECTIVE: J partial; g_c = 2 w_c (H_c - Ht_c) on the mask, zero elsewhere and
  // for x >= nx (the padding); the forward stage 0 of the adjoint source runs on g
  const float wc = a.w[c];
  double jacc = 0.0;
  int mine = 0;
  xdit0<L>(tile, tw, [&](int, int j, int line, cx<float>* v) {
    const int ra = row0 + 2 * line, rb = ra + 1;
    constexpr int R = StageShape<L, 0>::R, M = StageShape<L, 0>::M;
#pragma unroll
    for (int q = 0; q < R; q++) {
      const int x = j + q * M;
      float g[2] = {0.0f, 0.0f};
      if (x < a.nx) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
          const int row = ra + h;
          if (row >= a.rows) continue;
          const long long o = (long long)row * a.nx + x;
          const float hv = h ? v[q].y : v[q].x;
          if (a.H) a.H[c * a.H_cstride + o] = hv;
          if (wc != 0.0f && a.mask[o]) {
            mine = 1;
            const float r = hv - (a.Ht ? a.Ht[c * a.Ht_cstride + o] : a.Htc[c]);
            jacc += (double)wc * (double)r * (double)r;
            g[h] = 2.0f * wc * r;
          }
        }
      }
      v[q] = mk(g[0], g[1]);
    }
    return true;
  });
  for (int off = 16; off > 0; off >>= 1) jacc += __shfl_xor_sync(0xffffffffu, jacc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = jacc;
  const int any_mask = __syncthreads_or(mine);
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNT / 32; w++) s += red[w];
    a.Jpart[jc * gridDim.x + blockIdx.x] = s;
  }
  if (a.Jcount) finish_j(a);
  if (!a.adj_out) return;
  cx<float>* adj = reinterpret_cast<cx<float>*>(a.adj_out) + a.in_slot[jc] * a.in_cstride;
  if (!any_mask) {  // the adjoint source vanishes on all rows of this block
    for (int i = threadIdx.x; i < ROWS * a.P; i += kNT) {
      const int rr = i / a.P, k = i - rr * a.P, row = row0 + rr;
      if (row < a.rows) adj[(long long)row * a.P + k] = zero<float>();
    }
    return;
  }
  DifRange<float, L, kNT, 1, S, true>::run(tile, tw);
  xseparate<L>(tile, a.P, [&](int rr, int k, cx<float> v) {
    const int row = row0 + rr;
    if (row < a.rows) adj[(long long)row * a.P + k] = v;
  });
  }
  }
}

template <int L>
size_t xsmem() {
  return (size_t)(L + L * TB) * sizeof(float2);
}

template <int L, int SRC>
int run_xfwd_src(const XFwdArgs& a, int ncomp, cudaStream_t s) {
  const size_t sm = xsmem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xfwd<L, SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = true;
  }
  const int tiles = (a.rows + ROWS - 1) / ROWS;
  if (tiles == 0 || ncomp == 0) return 0;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  const int per_comp = (2 * nsm + ncomp - 1) / ncomp;  // two resident blocks per SM in total
  const int blocks = tiles < per_comp ? tiles : per_comp;
  k_xfwd<L, SRC><<<dim3(blocks, ncomp), kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
template <int L>
int run_xfwd(const XFwdArgs& a, int ncomp, cudaStream_t s) {
  if (a.src == SRC_RHO_POW) return run_xfwd_src<L, SRC_RHO_POW>(a, ncomp, s);
  if (a.src == SRC_RHO_M0) return run_xfwd_src<L, SRC_RHO_M0>(a, ncomp, s);
  return run_xfwd_src<L, SRC_VECTOR>(a, ncomp, s);
}
template <int L, int SINK, int MINB>
int run_xinv_sink(const XInvArgs& a, cudaStream_t s) {
  const size_t sm = xsmem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xinv<L, SINK, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  const int blocks = (a.rows - a.row_base + ROWS - 1) / ROWS;
  if (blocks <= 0 || a.ncomp == 0) return 0;
  const int gy = SINK == SINK_CHAIN ? 1 : a.ncomp;
  k_xinv<L, SINK, MINB><<<dim3(blocks, gy), kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
template <int L>
int run_xinv(const XInvArgs& a, cudaStream_t s) {
  if (a.sink == SINK_FIELD) return run_xinv_sink<L, SINK_FIELD, 2>(a, s);
  if (a.sink == SINK_OBJECTIVE) return run_xinv_sink<L, SINK_OBJECTIVE, 2>(a, s);
  if (a.ncomp == 1 && a.M0v == nullptr) return run_xinv_sink<L, SINK_CHAIN, 2>(a, s);  // contracted slot
  return run_xinv_sink<L, SINK_CHAIN, 1>(a, s);
}

}  // namespace

int xinv_rows_per_block() { return ROWS; }

int launch_xfwd(int L, const XFwdArgs& a, int ncomp, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_xfwd<LL>(a, ncomp, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}
int launch_xinv(int L, const XInvArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_xinv<LL>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

}  // namespace tmk
