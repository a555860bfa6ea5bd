// x-axis passes of the stray-field convolution (Sec. "Discretization", Eq. (convolution)).
//
// Forward: real rows (rho^p, rho^p M0_c of Sec. "Methodology" Eq. 2, or a given
// vector component) are zero padded from nx to L (implicitly: the first DIF
// stage reads only x < nx) and transformed two rows at a time (row a + i row b),
// then separated into the half spectra kx = 0..L/2. One block per (32-row tile,
// component).
// Inverse: half spectra are extended by Hermitian symmetry, two rows are
// recovered from one complex inverse transform, cropped to nx, and handed to a
// sink: write H; the least-squares objective and dJ/dH fused with the forward x
// transform of the adjoint source (per component: both are separable in c); or
// the chain rule dJ/drho = p rho^(p-1) M0 . (D g) (Sec. "Methodology",
// Eqs. (adjoint1)-(adjoint2)).
#include "fft.cuh"
#include "internal.h"

namespace tmk {

namespace {

constexpr int ROWS = 2 * TB;  // real rows per block
constexpr int CK = 32;        // kx columns per output chunk
constexpr int CKP = CK + 1;   // odd pitch of the chunk staging

template <int L>
struct XSmem {
  static constexpr int SP = (L / 2) | 1;  // odd pitch of a staged real row (>= nx)
  static constexpr size_t base = (size_t)(L + L * TB + 2 * TB * CKP) * sizeof(float2);
  static constexpr size_t rows = (size_t)ROWS * SP * sizeof(float);
};

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

// Forward x transform of 2*TB staged real rows (stage[rr * SP + x], x < nx) and
// write of the half spectra through out(rr, k, value) for k < P (zero beyond L/2).
template <int L, typename OUT>
__device__ __forceinline__ void xfwd_from_stage(cx<float>* tile, const cx<float>* tw, const float* stage, int nx,
                                                int P, cx<float>* chA, cx<float>* chB, OUT out) {
  constexpr int SP = XSmem<L>::SP;
  constexpr int S = plan_stages(L);
  dif_stage0_load<float, L, kNT>(tile, tw, [&](int pos, int line) {
    return pos < nx ? mk(stage[(2 * line) * SP + pos], stage[(2 * line + 1) * SP + pos]) : zero<float>();
  });
  __syncthreads();
  DifRange<float, L, kNT, 1, S>::run(tile, tw);
  for (int k0 = 0; k0 < P; k0 += CK) {
    for (int i = threadIdx.x; i < TB * CK; i += kNT) {
      const int line = i % TB, kk = i / TB, k = k0 + kk;
      cx<float> A = zero<float>(), B = zero<float>();
      if (k <= L / 2) {
        const cx<float> Z = tile[pos_of_k<L>(k) * TB + line];
        const cx<float> Zm = tile[pos_of_k<L>((L - k) % L) * TB + line];
        A = mk(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));  // (Z + conj Zm) / 2
        B = mk(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));  // (Z - conj Zm) / 2i
      }
      chA[line * CKP + kk] = A;
      chB[line * CKP + kk] = B;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * CK; i += kNT) {
      const int rr = i / CK, kk = i % CK, k = k0 + kk;
      if (k < P) out(rr, k, (rr & 1) ? chB[(rr >> 1) * CKP + kk] : chA[(rr >> 1) * CKP + kk]);
    }
    __syncthreads();
  }
}

// Inverse x transform of the spectra of 2*TB rows (slot pointer `in`, row pitch P)
// into staged real rows dst[rr * SP + x], x < nx.
template <int L>
__device__ __forceinline__ void xinv_to_stage(cx<float>* tile, const cx<float>* tw, const cx<float>* in, int row0,
                                              int rows, int nx, int P, cx<float>* chA, cx<float>* chB, float* dst) {
  constexpr int SP = XSmem<L>::SP;
  constexpr int S = plan_stages(L);
  for (int k0 = 0; k0 <= L / 2; k0 += CK) {
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * CK; i += kNT) {
      const int rr = i / CK, kk = i % CK, k = k0 + kk, row = row0 + rr;
      cx<float> v = zero<float>();
      if (row < rows && k <= L / 2) v = in[(long long)row * P + k];
      ((rr & 1) ? chB : chA)[(rr >> 1) * CKP + kk] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TB * CK; i += kNT) {
      const int line = i % TB, kk = i / TB, k = k0 + kk;
      if (k > L / 2) continue;
      const cx<float> A = chA[line * CKP + kk], B = chB[line * CKP + kk];
      if (k == 0 || k == L / 2) {
        tile[pos_of_k<L>(k) * TB + line] = mk(A.x, B.x);
      } else {
        tile[pos_of_k<L>(k) * TB + line] = mk(A.x - B.y, A.y + B.x);      // A + iB
        tile[pos_of_k<L>(L - k) * TB + line] = mk(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
      }
    }
  }
  __syncthreads();
  DitRange<float, L, kNT, 1, S>::run(tile, tw);
  dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
    if (pos < nx) {
      dst[(2 * line) * SP + pos] = v.x;
      dst[(2 * line + 1) * SP + pos] = v.y;
    }
  });
  __syncthreads();
}

template <int L>
__global__ void __launch_bounds__(kNT, 2) k_xfwd(XFwdArgs a) {
  constexpr int SP = XSmem<L>::SP;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  cx<float>* chA = tile + L * TB;
  cx<float>* chB = chA + TB * CKP;
  float* stage = reinterpret_cast<float*>(chB + TB * CKP);
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);

  const int row0 = blockIdx.x * ROWS;
  const int c = a.comp[blockIdx.y];
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[blockIdx.y] * a.out_cstride;
  for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
    const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
    float v = 0.0f;
    if (row < a.rows) {
      const long long o = (long long)row * a.nx + x;
      if (a.src == SRC_VECTOR) {
        v = a.vec[c * a.vec_cstride + o];
      } else {
        v = ipow(a.rho[o], a.p);
        if (a.src == SRC_RHO_M0) v *= a.M0v[c * a.M0v_cstride + o];
      }
    }
    stage[rr * SP + x] = v;
  }
  __syncthreads();
  xfwd_from_stage<L>(tile, tw, stage, a.nx, a.P, chA, chB, [&](int rr, int k, cx<float> v) {
    const int row = row0 + rr;
    if (row < a.rows) out[(long long)row * a.P + k] = v;
  });
}

template <int L>
__global__ void __launch_bounds__(kNT, 2) k_xinv(XInvArgs a) {
  constexpr int SP = XSmem<L>::SP;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  cx<float>* chA = tile + L * TB;
  cx<float>* chB = chA + TB * CKP;
  float* rows = reinterpret_cast<float*>(chB + TB * CKP);  // [ROWS][SP]
  float* acc = rows + ROWS * SP;                            // [ROWS][SP], CHAIN with ncomp > 1
  __shared__ double red[kNT / 32];
  __shared__ int any_mask;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int row0 = blockIdx.x * ROWS;
  const cx<float>* in0 = reinterpret_cast<const cx<float>*>(a.in);

  if (a.sink == SINK_CHAIN) {
    for (int j = 0; j < a.ncomp; j++) {
      xinv_to_stage<L>(tile, tw, in0 + a.in_slot[j] * a.in_cstride, row0, a.rows, a.nx, a.P, chA, chB, rows);
      if (a.ncomp > 1) {  // acc += M0_c . D_c (varying M0, uncontracted slots)
        for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
          const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
          float m = 0.0f;
          if (row < a.rows) m = a.M0v[a.comp[j] * a.M0v_cstride + (long long)row * a.nx + x];
          const float t = m * rows[rr * SP + x];
          acc[rr * SP + x] = (j == 0) ? t : acc[rr * SP + x] + t;
        }
      }
    }
    const float* dot = a.ncomp > 1 ? acc : rows;
    float gm = 0.0f;
    for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
      const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
      if (row >= a.rows) continue;
      const long long o = (long long)row * a.nx + x;
      const float G = dpow(a.rho[o], a.p) * dot[rr * SP + x];
      a.G[o] = G;
      gm = fmaxf(gm, fabsf(G));
    }
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((threadIdx.x & 31) == 0 && gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    return;
  }

  const int j = blockIdx.y, c = a.comp[j];
  const cx<float>* in = in0 + a.in_slot[j] * a.in_cstride;
  xinv_to_stage<L>(tile, tw, in, row0, a.rows, a.nx, a.P, chA, chB, rows);

  if (a.sink == SINK_FIELD) {
    for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
      const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
      if (row < a.rows) a.H[c * a.H_cstride + (long long)row * a.nx + x] = rows[rr * SP + x];
    }
    return;
  }

  // SINK_OBJECTIVE: J partial and g_c = 2 w_c (H_c - Ht_c) on the mask, in place in rows
  const float wc = a.w[c];
  if (threadIdx.x == 0) any_mask = 0;
  __syncthreads();
  double jacc = 0.0;
  int mine = 0;
  for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
    const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
    float g = 0.0f;
    if (row < a.rows) {
      const long long o = (long long)row * a.nx + x;
      const float h = rows[rr * SP + x];
      if (a.H) a.H[c * a.H_cstride + o] = h;
      if (wc != 0.0f && a.mask[o]) {
        mine = 1;
        const float r = h - (a.Ht ? a.Ht[c * a.Ht_cstride + o] : a.Htc[c]);
        jacc += (double)wc * (double)r * (double)r;
        g = 2.0f * wc * r;
      }
    }
    rows[rr * SP + x] = g;
  }
  for (int off = 16; off > 0; off >>= 1) jacc += __shfl_xor_sync(0xffffffffu, jacc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = jacc;
  if (mine) any_mask = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNT / 32; w++) s += red[w];
    a.Jpart[j * gridDim.x + blockIdx.x] = s;
  }
  if (!a.adj_out) return;
  cx<float>* adj = reinterpret_cast<cx<float>*>(a.adj_out) + a.in_slot[j] * a.in_cstride;
  if (!any_mask) {  // the adjoint source vanishes on all rows of this block
    for (int i = threadIdx.x; i < ROWS * a.P; i += kNT) {
      const int rr = i / a.P, k = i - rr * a.P, row = row0 + rr;
      if (row < a.rows) adj[(long long)row * a.P + k] = zero<float>();
    }
    return;
  }
  xfwd_from_stage<L>(tile, tw, rows, a.nx, a.P, chA, chB, [&](int rr, int k, cx<float> v) {
    const int row = row0 + rr;
    if (row < a.rows) adj[(long long)row * a.P + k] = v;
  });
}

template <int L>
int run_xfwd(const XFwdArgs& a, int ncomp, cudaStream_t s) {
  const size_t sm = XSmem<L>::base + XSmem<L>::rows;
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xfwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = true;
  }
  const int blocks = (a.rows + ROWS - 1) / ROWS;
  if (blocks == 0 || ncomp == 0) return 0;
  k_xfwd<L><<<dim3(blocks, ncomp), kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
template <int L>
int run_xinv(const XInvArgs& a, cudaStream_t s) {
  const size_t smax = XSmem<L>::base + 2 * XSmem<L>::rows;
  const size_t sm = XSmem<L>::base + ((a.sink == SINK_CHAIN && a.ncomp > 1) ? 2 : 1) * XSmem<L>::rows;
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xinv<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax) != cudaSuccess)
      return -1;
    init = true;
  }
  const int blocks = (a.rows + ROWS - 1) / ROWS;
  if (blocks == 0 || a.ncomp == 0) return 0;
  const int gy = a.sink == SINK_CHAIN ? 1 : a.ncomp;
  k_xinv<L><<<dim3(blocks, gy), kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
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
