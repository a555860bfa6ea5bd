// Small kernels: deterministic float64 objective reduction, max |G| and the
// box-constrained projected-gradient update rho <- clip(rho - alpha G / max|G|, 0, 1)
// (box constraint 0 <= rho <= 1 of Sec. "Methodology", after Eq. 1).
#include <stdint.h>

#include <mutex>

#include "../../include/topomag.h"
#include "internal.h"
#include "tma.cuh"

namespace tmk {

namespace {

// one block: fixed-order sum of the per-block partials
__global__ void k_j_finalize(const double* part, int n, double* J) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *J = red[0];
}

__global__ void k_absmax(const float* G, long long n, unsigned int* gmax) {
  __shared__ float wm[32];
  float m = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(G[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {  // one atomic per block
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, wm[w]);
    if (m > 0.0f) atomicMax(gmax, __float_as_uint(m));
  }
}

__global__ void k_update(float* rho, const float* G, long long n, float alpha, int normalize,
                         const unsigned int* gmax) {
  float step = alpha;
  if (normalize) {
    const float gm = __uint_as_float(*gmax);
    if (!(gm > 0.0f)) return;  // max|G| = 0: no update
    step = alpha / gm;
  }
  const bool aligned = ((reinterpret_cast<unsigned long long>(rho) | reinterpret_cast<unsigned long long>(G)) & 15ULL) == 0;
  const long long n4 = aligned ? n / 4 : 0;
  float4* r4 = reinterpret_cast<float4*>(rho);
  const float4* g4 = reinterpret_cast<const float4*>(G);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
    float4 r = r4[i];
    const float4 g = g4[i];
    r.x = fminf(fmaxf(r.x - step * g.x, 0.0f), 1.0f);
    r.y = fminf(fmaxf(r.y - step * g.y, 0.0f), 1.0f);
    r.z = fminf(fmaxf(r.z - step * g.z, 0.0f), 1.0f);
    r.w = fminf(fmaxf(r.w - step * g.w, 0.0f), 1.0f);
    r4[i] = r;
  }
  for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
    rho[i] = fminf(fmaxf(rho[i] - step * G[i], 0.0f), 1.0f);
}

__global__ void k_scale(float* dst, const float* src, long long n, float coef) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = coef * src[i];
}

// [zlo, zhi) of the planes that hold a nonzero mask entry (ext preset to (INT_MAX-ish, 0))
__global__ void k_mask_extent(const uint8_t* mask, int nz, long long plane, int* ext) {
  for (int z = blockIdx.y; z < nz; z += gridDim.y) {
    const uint8_t* m = mask + (long long)z * plane;
    int any = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane && !any;
         i += (long long)gridDim.x * blockDim.x)
      any = m[i] != 0;
    any = __syncthreads_or(any);
    if (any && threadIdx.x == 0) {
      atomicMin(&ext[0], z);
      atomicMax(&ext[1], z + 1);
    }
  }
}

int grid_for(long long n, int per) {
  long long b = (n + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 152 * 8) b = 152 * 8;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Scratch of tm_optimize_step_noalloc, a file-scope device array instead of an
// allocation: slot 0 receives max|G|, slots 1..nb the maxima of the nb slices
// of kNoallocSlice elements. Every call overwrites the slots it reads.
constexpr int kNoallocSlice = 2048;
constexpr int kNoallocMaxSlices = 16384;
static __device__ __align__(256) float g_noalloc_scratch[1 + kNoallocMaxSlices];

__global__ void k_slice_absmax(const float* G, long long n, float* scratch) {
  __shared__ float red[8];
  const long long base = (long long)blockIdx.x * kNoallocSlice;
  float m = 0.0f;
  for (int i = threadIdx.x; i < kNoallocSlice; i += blockDim.x) {
    const long long k = base + i;
    if (k < n) m = fmaxf(m, fabsf(G[k]));
  }
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, red[w]);
    scratch[1 + blockIdx.x] = m;
  }
}

__global__ void k_reduce_slices(float* scratch, int nb) {
  __shared__ float red[8];
  float m = 0.0f;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmaxf(m, scratch[1 + i]);
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, red[w]);
    scratch[0] = m;
  }
}

// ---------------------------------------------------------------------------
// Validation of rho (box constraint 0 <= rho <= 1, Sec. "Methodology"): count of
// entries that are NaN or outside [0, 1] (integer count, any order gives the same).
__global__ void k_check_design(const float* rho, long long n, unsigned long long* bad) {
  unsigned c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c += !(rho[i] >= 0.0f && rho[i] <= 1.0f);  // NaN fails both comparisons
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, (unsigned long long)c);
}

// Per-block float64 partials of sum rho and of the count of intermediate densities
// 0.1 < rho < 0.9 (the quantities of Figs. 4 and 3), grid-stride in a fixed
// assignment; k_rho_stats_final sums them in block order.
__global__ void k_rho_stats(const float* rho, long long n, double* part) {
  __shared__ double rs[256], rc[256];
  double s = 0.0, c = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = rho[i];
    s += (double)r;
    c += (r > 0.1f && r < 0.9f) ? 1.0 : 0.0;
  }
  rs[threadIdx.x] = s;
  rc[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      rs[threadIdx.x] += rs[threadIdx.x + w];
      rc[threadIdx.x] += rc[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rs[0];
    part[2 * blockIdx.x + 1] = rc[0];
  }
}
__global__ void k_rho_stats_final(const double* part, int nblk, double* out) {
  if (threadIdx.x == 0) {
    double s = 0.0, c = 0.0;
    for (int b = 0; b < nblk; b++) {
      s += part[2 * b];
      c += part[2 * b + 1];
    }
    out[0] = s;
    out[1] = c;
  }
}

// Self-test of the bounded mbarrier wait: the barrier expects one arrival that never
// comes, so the wait runs out after `polls` polls, flags the status word and returns.
__global__ void k_wait_selftest(unsigned* status, int polls) {
  __shared__ __align__(8) unsigned long long mb;
  if (threadIdx.x == 0) {
    mbar_init(&mb, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_limit(&mb, 0, polls, status);
  __syncthreads();
}

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[256] = {nullptr};  // device address of g_noalloc_scratch, per device ordinal


// Quadratic stencil objective (Sec. "Optimization of field and gradient"): row k of
// a sparse matrix S picks a linear combination r_k = sum_e a_e H[idx_e] of field
// values; J = sum_k c_k r_k^2 (float64 block partials), then dJ/dH at every
// referenced value from the column form of S: sum over its rows of 2 c_k r_k a.
__global__ void k_stencil_rows(long long K, const long long* rp, const long long* idx, const double* a,
                               const double* c, const float* H, double* r, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < K; k += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (long long e = rp[k]; e < rp[k + 1]; e++) v += a[e] * (double)H[idx[e]];
    r[k] = v;
    s += c[k] * v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_stencil_cols(long long U, const long long* cp, const long long* cidx, const int* crow,
                               const double* ca, const double* c, const double* r, float* gH) {
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < U; u += (long long)gridDim.x * blockDim.x) {
    double g = 0.0;
    for (long long e = cp[u]; e < cp[u + 1]; e++) {
      const int k = crow[e];
      g += 2.0 * c[k] * r[k] * ca[e];
    }
    gH[cidx[u]] = (float)g;
  }
}
}  // namespace

int launch_stencil(const StencilArgs& a, cudaStream_t s) {
  k_stencil_rows<<<a.nblk, 256, 0, s>>>(a.K, a.rp, a.idx, a.a, a.c, a.H, a.r, a.part);
  k_j_finalize<<<1, 256, 0, s>>>(a.part, a.nblk, a.J);
  const long long b = (a.U + 255) / 256;
  k_stencil_cols<<<(int)(b < 1 ? 1 : (b > 4096 ? 4096 : b)), 256, 0, s>>>(a.U, a.cp, a.cidx, a.crow, a.ca, a.c, a.r,
                                                                         a.gH);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_scale(float* dst, const float* src, long long n, float coef, cudaStream_t s) {
  k_scale<<<grid_for(n, 256 * 8), 256, 0, s>>>(dst, src, n, coef);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
int launch_check_design(const float* rho, long long n, unsigned long long* bad, cudaStream_t s) {
  k_check_design<<<grid_for(n, 256 * 8), 256, 0, s>>>(rho, n, bad);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
int launch_rho_stats(const float* rho, long long n, double* part, int nblk, double* out, cudaStream_t s) {
  k_rho_stats<<<nblk, 256, 0, s>>>(rho, n, part);
  k_rho_stats_final<<<1, 32, 0, s>>>(part, nblk, out);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
int launch_wait_selftest(unsigned* status, int polls, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(status, polls);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

int launch_j_finalize(const double* part, int n, double* J, cudaStream_t s) {
  k_j_finalize<<<1, 256, 0, s>>>(part, n, J);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
int launch_mask_extent(const uint8_t* mask, int nz, long long plane, int* ext, cudaStream_t s) {
  if (cudaMemsetAsync(ext, 0x7f, sizeof(int), s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(ext + 1, 0, sizeof(int), s) != cudaSuccess) return -1;
  const int gx = (int)((plane + 1023) / 1024 < 8 ? (plane + 1023) / 1024 : 8);
  k_mask_extent<<<dim3(gx, nz < 65535 ? nz : 65535), 256, 0, s>>>(mask, nz, plane, ext);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
int launch_absmax(const float* G, long long n, unsigned int* gmax, cudaStream_t s) {
  k_absmax<<<grid_for(n, 256 * 8), 256, 0, s>>>(G, n, gmax);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}
int launch_update(float* rho, const float* G, long long n, float alpha, int normalize, const unsigned int* gmax,
                  cudaStream_t s) {
  k_update<<<grid_for(n / 4 + 1, 256 * 4), 256, 0, s>>>(rho, G, n, alpha, normalize, gmax);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tmk

// A context-free projected-gradient step for callers that may not allocate
// device memory. See include/topomag.h. The paper has no counterpart: this is
// an interface convenience, not part of the method.
extern "C" int tm_optimize_step_noalloc(float* rho, const float* dJdrho, long long n, float alpha, int normalize,
                                        void* stream) {
  using namespace tmk;
  if (!rho || !dJdrho || n < 0 || !isfinite(alpha)) return TM_ERR_ARG;
  if (n > (long long)kNoallocSlice * kNoallocMaxSlices) return TM_ERR_SIZE;
  if (n == 0) return TM_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return TM_ERR_CUDA;
  float* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // once per device, with that device current: the host-side name of the
      // array is not a device address; ask the runtime for the real one
      if (cudaGetSymbolAddress(reinterpret_cast<void**>(&g_noalloc_ptr[dev]), g_noalloc_scratch) != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        return TM_ERR_CUDA;
      }
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (normalize) {
    const int nb = (int)((n + kNoallocSlice - 1) / kNoallocSlice);
    k_slice_absmax<<<nb, 256, 0, s>>>(dJdrho, n, scratch);
    k_reduce_slices<<<1, 256, 0, s>>>(scratch, nb);
    if (cudaPeekAtLastError() != cudaSuccess) return TM_ERR_CUDA;
  }
  // the update kernel of tm_optimize_step reads max|G| as float bits from slot 0
  if (launch_update(rho, dJdrho, n, alpha, normalize, reinterpret_cast<const unsigned int*>(scratch), s) != 0)
    return TM_ERR_CUDA;
  return TM_OK;
}
