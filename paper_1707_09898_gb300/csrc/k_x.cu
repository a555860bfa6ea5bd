// x-axis passes of the stray-field convolution (Sec. "Discretization", Eq. (convolution)).
//
// Forward: real rows (rho^p M0 of Sec. "Methodology" Eq. 2, or a given vector
// field) are zero padded from nx to L (implicitly: the first DIF stage reads
// only x < nx) and transformed two rows at a time (row a + i row b), then
// separated into the half spectra kx = 0..L/2.
// Inverse: half spectra are extended by Hermitian symmetry, two rows are
// recovered from one complex inverse transform, cropped to nx, and handed to a
// sink: write H; or the least-squares objective and dJ/dH fused with the
// forward x transform of the adjoint source; or the chain rule
// dJ/drho = p rho^(p-1) M0 . (D g) (Sec. "Methodology", Eqs. (adjoint1)-(adjoint2)).
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
  const int nfft = a.src == SRC_RHO_CONST ? 1 : 3;
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out);
  for (int c = 0; c < nfft; c++) {
    for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
      const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
      float v = 0.0f;
      if (row < a.rows) {
        const long long o = (long long)row * a.nx + x;
        if (a.src == SRC_VECTOR) {
          v = a.vec[c * a.vec_cstride + o];
        } else {
          v = ipow(a.rho[o], a.p);
          if (a.src == SRC_RHO_FIELD) v *= a.M0v[c * a.M0v_cstride + o];
        }
      }
      stage[rr * SP + x] = v;
    }
    __syncthreads();
    xfwd_from_stage<L>(tile, tw, stage, a.nx, a.P, chA, chB, [&](int rr, int k, cx<float> v) {
      const int row = row0 + rr;
      if (row >= a.rows) return;
      const long long o = (long long)row * a.P + k;
      if (a.src == SRC_RHO_CONST) {
#pragma unroll
        for (int cc = 0; cc < 3; cc++) out[cc * a.out_cstride + o] = scale(v, a.M0c[cc]);
      } else {
        out[c * a.out_cstride + o] = v;
      }
    });
  }
}

template <int L>
__global__ void __launch_bounds__(kNT, 1) k_xinv(XInvArgs a) {
  constexpr int SP = XSmem<L>::SP;
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  cx<float>* chA = tile + L * TB;
  cx<float>* chB = chA + TB * CKP;
  float* rout = reinterpret_cast<float*>(chB + TB * CKP);  // [3][ROWS][SP]
  __shared__ double red[kNT / 32];
  __shared__ int any_mask;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);

  const int row0 = blockIdx.x * ROWS;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.in);
  for (int c = 0; c < 3; c++) {
    // Hermitian extension of the two rows of each line, placed at DIF positions
    for (int k0 = 0; k0 <= L / 2; k0 += CK) {
      __syncthreads();
      for (int i = threadIdx.x; i < ROWS * CK; i += kNT) {
        const int rr = i / CK, kk = i % CK, k = k0 + kk, row = row0 + rr;
        cx<float> v = zero<float>();
        if (row < a.rows && k <= L / 2) v = in[c * a.in_cstride + (long long)row * a.P + k];
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
    float* rc = rout + c * ROWS * SP;
    dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
      if (pos < a.nx) {
        rc[(2 * line) * SP + pos] = v.x;
        rc[(2 * line + 1) * SP + pos] = v.y;
      }
    });
    __syncthreads();
  }

  if (a.sink == SINK_FIELD) {
    for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
      const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
      if (row >= a.rows) continue;
      const long long o = (long long)row * a.nx + x;
#pragma unroll
      for (int c = 0; c < 3; c++) a.H[c * a.H_cstride + o] = rout[c * ROWS * SP + rr * SP + x];
    }
    return;
  }

  if (a.sink == SINK_CHAIN) {
    float gm = 0.0f;
    for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
      const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
      if (row >= a.rows) continue;
      const long long o = (long long)row * a.nx + x;
      float m0x = a.M0c[0], m0y = a.M0c[1], m0z = a.M0c[2];
      if (a.M0v) {
        m0x = a.M0v[o];
        m0y = a.M0v[a.M0v_cstride + o];
        m0z = a.M0v[2 * a.M0v_cstride + o];
      }
      const float dot = m0x * rout[rr * SP + x] + m0y * rout[ROWS * SP + rr * SP + x] +
                        m0z * rout[2 * ROWS * SP + rr * SP + x];
      const float G = dpow(a.rho[o], a.p) * dot;
      a.G[o] = G;
      gm = fmaxf(gm, fabsf(G));
    }
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((threadIdx.x & 31) == 0 && gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    return;
  }

  // SINK_OBJECTIVE: J partial, g = 2 w (H - Ht) on the mask (in place in rout)
  if (threadIdx.x == 0) any_mask = 0;
  __syncthreads();
  double jacc = 0.0;
  int mine = 0;
  for (int i = threadIdx.x; i < ROWS * a.nx; i += kNT) {
    const int rr = i / a.nx, x = i - rr * a.nx, row = row0 + rr;
    float g[3] = {0.0f, 0.0f, 0.0f};
    if (row < a.rows) {
      const long long o = (long long)row * a.nx + x;
      if (a.H) {
#pragma unroll
        for (int c = 0; c < 3; c++) a.H[c * a.H_cstride + o] = rout[c * ROWS * SP + rr * SP + x];
      }
      if (a.mask[o]) {
        mine = 1;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const float ht = a.Ht ? a.Ht[c * a.Ht_cstride + o] : a.Htc[c];
          const float r = rout[c * ROWS * SP + rr * SP + x] - ht;
          jacc += (double)a.w[c] * (double)r * (double)r;
          g[c] = 2.0f * a.w[c] * r;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) rout[c * ROWS * SP + rr * SP + x] = g[c];
  }
  for (int off = 16; off > 0; off >>= 1) jacc += __shfl_xor_sync(0xffffffffu, jacc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = jacc;
  if (mine) any_mask = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kNT / 32; w++) s += red[w];
    a.Jpart[blockIdx.x] = s;
  }
  cx<float>* adj = reinterpret_cast<cx<float>*>(a.adj_out);
  if (!any_mask) {  // the adjoint source vanishes on all rows of this block
    for (int i = threadIdx.x; i < ROWS * a.P; i += kNT) {
      const int rr = i / a.P, k = i - rr * a.P, row = row0 + rr;
      if (row >= a.rows) continue;
#pragma unroll
      for (int c = 0; c < 3; c++) adj[c * a.in_cstride + (long long)row * a.P + k] = zero<float>();
    }
    return;
  }
  for (int c = 0; c < 3; c++) {
    xfwd_from_stage<L>(tile, tw, rout + c * ROWS * SP, a.nx, a.P, chA, chB, [&](int rr, int k, cx<float> v) {
      const int row = row0 + rr;
      if (row < a.rows) adj[c * a.in_cstride + (long long)row * a.P + k] = v;
    });
  }
}

template <int L>
size_t xfwd_smem() {
  return (size_t)(L + L * TB + 2 * TB * CKP) * sizeof(float2) + (size_t)ROWS * XSmem<L>::SP * sizeof(float);
}
template <int L>
size_t xinv_smem() {
  return (size_t)(L + L * TB + 2 * TB * CKP) * sizeof(float2) + (size_t)3 * ROWS * XSmem<L>::SP * sizeof(float);
}

template <int L>
int run_xfwd(const XFwdArgs& a, cudaStream_t s) {
  const size_t sm = xfwd_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xfwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = true;
  }
  const int blocks = (a.rows + ROWS - 1) / ROWS;
  if (blocks == 0) return 0;
  k_xfwd<L><<<blocks, kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
template <int L>
int run_xinv(const XInvArgs& a, cudaStream_t s) {
  const size_t sm = xinv_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xinv<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = true;
  }
  const int blocks = (a.rows + ROWS - 1) / ROWS;
  if (blocks == 0) return 0;
  k_xinv<L><<<blocks, kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int xinv_rows_per_block() { return ROWS; }

int launch_xfwd(int L, const XFwdArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_xfwd<LL>(a, s);
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
