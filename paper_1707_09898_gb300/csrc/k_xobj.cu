// The objective on the target rows (Sec. "Methodology", the objective of Eq. (1),
// here J = sum_mask sum_c w_c (H_c - Ht_c)^2) for the prepared path, with its
// partial derivative g = 2 w_c (H_c - Ht_c) transformed back along x:
//   half spectra of two real rows -> inverse x transform -> H, J, g -> forward x
//   transform of g -> half spectra of the adjoint source.
// The target rows are few (one or a few planes), so this kernel is bound by latency,
// not bandwidth: a group of four warps per pair of rows runs an iterative mixed-radix
// Stockham transform (radix 4, 2, 3 stages in natural order, loops rather than
// unrolled stages) in its own shared-memory buffers, synchronising only the group
// (named barrier). The code is a few hundred instructions for every length.
#include "fft.cuh"
#include "internal.h"

namespace tmk {

namespace {

constexpr int OW = 8;   // warps per block
constexpr int GW = 4;   // warps per row pair (one transform group)
constexpr int GT = GW * 32;
constexpr int NG = OW / GW;  // row pairs per block
constexpr int KI = 3;   // ceil((576 / 2 + 1) / GT): half-spectrum values per thread
constexpr int XI = 5;   // ceil(576 / GT): real values per thread

__device__ __forceinline__ cx<float> cmul(cx<float> a, cx<float> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ cx<float> conjf(cx<float> a) { return mk(a.x, -a.y); }

// barrier of the GT threads of transform group g (ids 1.. ; 0 is the block barrier)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(GT) : "memory"); }
__device__ __forceinline__ void group_sync8(int g) { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(64) : "memory"); }

// One group: length-L transform of src into dst (natural order both), sign -1 forward,
// +1 inverse (unnormalised). Stockham stages: for j < L/R, the R inputs src[j + r L/R]
// times W^(r (j mod Ns) L/(Ns R)) go through a radix-R DFT to dst[(j/Ns) Ns R + j mod
// Ns + r Ns], Ns the product of the radices before. Returns the buffer holding the result.
__device__ cx<float>* group_fft(cx<float>* src, cx<float>* dst, int L, const cx<float>* tw, bool inverse, int gt,
                                int g) {
  int rem = L, Ns = 1;
  while (rem > 1) {
    const int R = rem % 4 == 0 ? 4 : (rem % 2 == 0 ? 2 : 3);
    const int M = L / R;
    const int step = L / (Ns * R);
#pragma unroll 1
    for (int j = gt; j < M; j += GT) {
      const int k = j % Ns;
      cx<float> v[4];
#pragma unroll
      for (int r = 0; r < 4; r++)
        if (r < R) {
          v[r] = src[j + r * M];
          if (r > 0 && k > 0) {
            cx<float> w = tw[r * k * step];
            if (inverse) w = conjf(w);
            v[r] = cmul(v[r], w);
          }
        }
      cx<float> y[4];
      if (R == 2) {
        y[0] = v[0] + v[1];
        y[1] = v[0] - v[1];
      } else if (R == 4) {
        // y_q = sum_r v_r (-i)^(q r) forward, (+i)^(q r) inverse
        const cx<float> a = v[0] + v[2], b = v[0] - v[2], c = v[1] + v[3], d = v[1] - v[3];
        const cx<float> di = inverse ? mk(-d.y, d.x) : mk(d.y, -d.x);  // (+-i) d
        y[0] = a + c;
        y[2] = a - c;
        y[1] = b + di;
        y[3] = b - di;
      } else {  // R == 3: W3 = exp(-+2 pi i / 3) = -1/2 -+ i sqrt(3)/2
        const float h = 0.8660254037844386f;
        const cx<float> s = v[1] + v[2], t = v[1] - v[2];
        const cx<float> m = mk(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
        const cx<float> it = inverse ? mk(-h * t.y, h * t.x) : mk(h * t.y, -h * t.x);  // (+-i) h t
        y[0] = v[0] + s;
        y[1] = m + it;
        y[2] = m - it;
      }
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < 4; r++)
        if (r < R) dst[base + r * Ns] = y[r];
    }
    group_sync(g);
    cx<float>* t = src;
    src = dst;
    dst = t;
    Ns *= R;
    rem /= R;
  }
  return src;
}

__global__ void __launch_bounds__(OW * 32) k_xobj(XInvArgs a, int L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int any_mask[NG];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = warp / GW, gt = threadIdx.x - g * GT;
  cx<float>* b0 = tw + L + g * 2 * L;
  cx<float>* b1 = b0 + L;
  for (int i = threadIdx.x; i < L; i += OW * 32) tw[i] = reinterpret_cast<const cx<float>*>(a.tw)[i];
  if (gt == 0) any_mask[g] = 0;
  pdl_wait();  // the spectra, J partials and outputs belong to earlier kernels
  __syncthreads();
  const int jc = blockIdx.y, c = a.comp[jc];
  const float wc = a.w[c];
  const int K = L / 2 + 1;
  const int ra = a.row_base + (blockIdx.x * NG + g) * 2, rb = ra + 1;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.in) + a.in_slot[jc] * a.in_cstride;
  double jacc = 0.0;
  if (ra < a.rows) {  // uniform over the group
    const bool hb = rb < a.rows;
    // Z(k) = A(k) + i B(k) over the full length, A and B extended by Hermitian symmetry;
    // every load of the thread is issued before the first store
    cx<float> Av[KI], Bv[KI];
#pragma unroll
    for (int it = 0; it < KI; it++) {
      const int k = gt + GT * it;
      Av[it] = k < K ? in[(long long)ra * a.P + k] : zero<float>();
      Bv[it] = (k < K && hb) ? in[(long long)rb * a.P + k] : zero<float>();
    }
#pragma unroll
    for (int it = 0; it < KI; it++) {
      const int k = gt + GT * it;
      if (k < K) {
        const cx<float> A = Av[it], B = Bv[it];
        b0[k] = mk(A.x - B.y, A.y + B.x);
        if (k > 0 && k < L - k) b0[L - k] = mk(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
      }
    }
    group_sync(g);
    cx<float>* z = group_fft(b0, b1, L, tw, true, gt, g);
    cx<float>* o = z == b0 ? b1 : b0;
    // mask and target values of the thread's cells, all loads first
    unsigned char mk2[XI][2];
    float ht[XI][2];
#pragma unroll
    for (int it = 0; it < XI; it++) {
      const int x = gt + GT * it;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int row = h ? rb : ra;
        const bool ok = x < a.nx && (h == 0 || hb) && wc != 0.0f;
        const long long e = (long long)row * a.nx + x;
        mk2[it][h] = ok ? a.mask[e] : 0;
        ht[it][h] = (ok && a.Ht) ? a.Ht[c * a.Ht_cstride + e] : a.Htc[c];
      }
    }
    int mine = 0;
#pragma unroll
    for (int it = 0; it < XI; it++) {
      const int x = gt + GT * it;
      if (x < L) {
        float gv[2] = {0.0f, 0.0f};
        if (x < a.nx) {
          const cx<float> hv = z[x];
#pragma unroll
          for (int h = 0; h < 2; h++) {
            if (mk2[it][h]) {
              mine = 1;
              const float r = (h ? hv.y : hv.x) - ht[it][h];
              jacc += (double)wc * (double)r * (double)r;
              gv[h] = 2.0f * wc * r;
            }
          }
        }
        o[x] = mk(gv[0], gv[1]);
      }
    }
    if (mine) any_mask[g] = 1;
    group_sync(g);
    cx<float>* adj = reinterpret_cast<cx<float>*>(a.adj_out) + a.in_slot[jc] * a.in_cstride;
    if (!any_mask[g]) {  // no target cell on these rows: the adjoint source vanishes
      for (int k = gt; k < a.P; k += GT) {
        adj[(long long)ra * a.P + k] = zero<float>();
        if (hb) adj[(long long)rb * a.P + k] = zero<float>();
      }
    } else {
      cx<float>* Zg = group_fft(o, z, L, tw, false, gt, g);
      for (int k = gt; k < a.P; k += GT) {
        cx<float> A = zero<float>(), B = zero<float>();
        if (k < K) {
          const cx<float> Z = Zg[k], Zm = Zg[(L - k) % L];
          A = mk(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));  // (Z + conj Zm) / 2
          B = mk(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));  // (Z - conj Zm) / 2i
        }
        adj[(long long)ra * a.P + k] = A;
        if (hb) adj[(long long)rb * a.P + k] = B;
      }
    }
  }
  // J partial of the block in a fixed order, then the last block's sum
  for (int off = 16; off > 0; off >>= 1) jacc += __shfl_xor_sync(0xffffffffu, jacc, off);
  __shared__ double red[OW];
  if (lane == 0) red[warp] = jacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < OW; w++) s += red[w];
    a.Jpart[jc * gridDim.x + blockIdx.x] = s;
  }
  __shared__ unsigned int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(a.Jcount, 1u) == gridDim.x * gridDim.y - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double r2[OW * 32];
  const int n = gridDim.x * gridDim.y;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += OW * 32) s += __ldcg(a.Jpart + i);
  r2[threadIdx.x] = s;
  __syncthreads();
  for (int w = OW * 16; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) r2[threadIdx.x] += r2[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *a.Jout = r2[0];
    *a.Jcount = 0u;
  }
}

// ---------------------------------------------------------------------------
// L = 512 = 8^3: the same pass with the transform's stages fixed at compile time: three
// radix-8 Stockham stages (index arithmetic by shifts and masks, three group barriers per
// transform), a group of two warps per row pair, two row pairs per block.
constexpr int G8 = 64;          // threads per row pair
constexpr int NG8 = 2;          // row pairs per block (measured: 14.7 us per launch, 16.1 with 4)
constexpr int NT8 = G8 * NG8;   // threads per block

// Stockham stage s of a length-512 radix-8 transform: Ns = 8^s; thread j < 64 reads
// src[j + 64 r], twiddles by W^(r k 64 / Ns) (k = j mod Ns), DFT-8, writes
// dst[(j / Ns) 8 Ns + k + r Ns].
template <int S, bool INV>
__device__ __forceinline__ void r8_stage(const cx<float>* src, cx<float>* dst, const cx<float>* tw, int j) {
  constexpr int Ns = S == 0 ? 1 : (S == 1 ? 8 : 64);
  constexpr int step = 64 / Ns;
  const int k = j & (Ns - 1);
  cx<float> v[8];
#pragma unroll
  for (int r = 0; r < 8; r++) v[r] = src[j + 64 * r];
  if (S > 0 && k > 0) {
#pragma unroll
    for (int r = 1; r < 8; r++) {
      const cx<float> w = tw[r * k * step];
      v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
  }
  DftF<8, INV>::run(v);
  const int base = (j / Ns) * (8 * Ns) + k;
#pragma unroll
  for (int r = 0; r < 8; r++) dst[base + r * Ns] = v[r];
}
template <bool INV>
__device__ __forceinline__ cx<float>* r8_fft(cx<float>* b0, cx<float>* b1, const cx<float>* tw, int j, int g) {
  r8_stage<0, INV>(b0, b1, tw, j);
  group_sync8(g);
  r8_stage<1, INV>(b1, b0, tw, j);
  group_sync8(g);
  r8_stage<2, INV>(b0, b1, tw, j);
  group_sync8(g);
  return b1;
}

__global__ void __launch_bounds__(NT8) k_xobj512(XInvArgs a) {
  constexpr int L = 512, K = L / 2 + 1, KI8 = (K + G8 - 1) / G8, XI8 = L / G8;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int any_mask[NG8];
  __shared__ double red[NT8 / 32];
  __shared__ unsigned int last;
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  const int g = threadIdx.x / G8, gt = threadIdx.x - g * G8;
  cx<float>* b0 = tw + L + g * 2 * L;
  cx<float>* b1 = b0 + L;
  for (int i = threadIdx.x; i < L; i += NT8) tw[i] = reinterpret_cast<const cx<float>*>(a.tw)[i];
  if (gt == 0) any_mask[g] = 0;
  pdl_wait();  // the spectra, J partials and outputs belong to earlier kernels
  __syncthreads();
  const int jc = blockIdx.y, c = a.comp[jc];
  const float wc = a.w[c];
  const int ra = a.row_base + (blockIdx.x * NG8 + g) * 2, rb = ra + 1;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.in) + a.in_slot[jc] * a.in_cstride;
  double jacc = 0.0;
  if (ra < a.rows) {  // uniform over the group
    const bool hb = rb < a.rows;
    cx<float> Av[KI8], Bv[KI8];
    unsigned char mk2[XI8][2];
    float ht[XI8][2];
#pragma unroll
    for (int it = 0; it < KI8; it++) {
      const int k = gt + G8 * it;
      Av[it] = k < K ? in[(long long)ra * a.P + k] : zero<float>();
      Bv[it] = (k < K && hb) ? in[(long long)rb * a.P + k] : zero<float>();
    }
    // mask and target values of the thread's cells, loaded while the transform runs
#pragma unroll
    for (int it = 0; it < XI8; it++) {
      const int x = gt + G8 * it;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int row = h ? rb : ra;
        const bool ok = x < a.nx && (h == 0 || hb) && wc != 0.0f;
        const long long e = (long long)row * a.nx + x;
        mk2[it][h] = ok ? a.mask[e] : 0;
        ht[it][h] = (ok && a.Ht) ? a.Ht[c * a.Ht_cstride + e] : a.Htc[c];
      }
    }
#pragma unroll
    for (int it = 0; it < KI8; it++) {
      const int k = gt + G8 * it;
      if (k < K) {
        const cx<float> A = Av[it], B = Bv[it];
        b0[k] = mk(A.x - B.y, A.y + B.x);                                 // A + iB
        if (k > 0 && k < L - k) b0[L - k] = mk(A.x + B.y, B.x - A.y);  // conj(A) + i conj(B)
      }
    }
    group_sync8(g);
    const cx<float>* z = r8_fft<true>(b0, b1, tw, gt, g);  // in b1
    int mine = 0;
#pragma unroll
    for (int it = 0; it < XI8; it++) {
      const int x = gt + G8 * it;
      float gv[2] = {0.0f, 0.0f};
      if (x < a.nx) {
        const cx<float> hv = z[x];
#pragma unroll
        for (int h = 0; h < 2; h++) {
          if (mk2[it][h]) {
            mine = 1;
            const float r = (h ? hv.y : hv.x) - ht[it][h];
            jacc += (double)wc * (double)r * (double)r;
            gv[h] = 2.0f * wc * r;
          }
        }
      }
      b0[x] = mk(gv[0], gv[1]);
    }
    if (mine) any_mask[g] = 1;
    group_sync8(g);
    cx<float>* adj = reinterpret_cast<cx<float>*>(a.adj_out) + a.in_slot[jc] * a.in_cstride;
    if (!any_mask[g]) {  // no target cell on these rows: the adjoint source vanishes
      for (int k = gt; k < a.P; k += G8) {
        adj[(long long)ra * a.P + k] = zero<float>();
        if (hb) adj[(long long)rb * a.P + k] = zero<float>();
      }
    } else {
      const cx<float>* Zg = r8_fft<false>(b0, b1, tw, gt, g);
      for (int k = gt; k < a.P; k += G8) {
        cx<float> A = zero<float>(), B = zero<float>();
        if (k < K) {
          const cx<float> Z = Zg[k], Zm = Zg[(L - k) % L];
          A = mk(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));  // (Z + conj Zm) / 2
          B = mk(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));  // (Z - conj Zm) / 2i
        }
        adj[(long long)ra * a.P + k] = A;
        if (hb) adj[(long long)rb * a.P + k] = B;
      }
    }
  }
  // J partial of the block in a fixed order, then the last block's sum
  for (int off = 16; off > 0; off >>= 1) jacc += __shfl_xor_sync(0xffffffffu, jacc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = jacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT8 / 32; w++) s += red[w];
    a.Jpart[jc * gridDim.x + blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(a.Jcount, 1u) == gridDim.x * gridDim.y - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double r2[NT8];
  const int n = gridDim.x * gridDim.y;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += NT8) s += __ldcg(a.Jpart + i);
  r2[threadIdx.x] = s;
  __syncthreads();
  for (int w = NT8 / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) r2[threadIdx.x] += r2[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *a.Jout = r2[0];
    *a.Jcount = 0u;
  }
}

}  // namespace

size_t xobj_smem(int L) { return (size_t)(L + NG * 2 * L) * sizeof(float2); }

int launch_xobj(int L, const XInvArgs& a, cudaStream_t s) {
  if (L == 512) {
    constexpr size_t sm8 = (size_t)(512 + NG8 * 2 * 512) * sizeof(float2);
    static bool init8 = false;
    if (!init8) {
      if (cudaFuncSetAttribute(k_xobj512, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm8) != cudaSuccess)
        return -1;
      init8 = true;
    }
    const int rows = a.rows - a.row_base;
    const int blocks = (rows + 2 * NG8 - 1) / (2 * NG8);
    if (blocks <= 0 || a.ncomp == 0) return 0;
    if (!a.Jcount || !a.adj_out) return -1;
    return launch_k(k_xobj512, dim3(blocks, a.ncomp), dim3(NT8), sm8, s, a.pdl != 0, a) == cudaSuccess ? 0 : -1;
  }
  const size_t sm = xobj_smem(L);
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xobj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xobj_smem(576)) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  const int rows = a.rows - a.row_base;
  const int blocks = (rows + 2 * NG - 1) / (2 * NG);
  if (blocks <= 0 || a.ncomp == 0 || !a.Jcount || !a.adj_out) return blocks <= 0 || a.ncomp == 0 ? 0 : -1;
  return launch_k(k_xobj, dim3(blocks, a.ncomp), dim3(OW * 32), sm, s, a.pdl != 0, a, L) == cudaSuccess ? 0 : -1;
}

int xobj_rows_per_block() { return 2 * (NG < NG8 ? NG : NG8); }  // the fewest rows any block holds

}  // namespace tmk
