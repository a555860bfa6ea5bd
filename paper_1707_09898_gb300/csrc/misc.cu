// Small kernels: deterministic float64 objective reduction, max |G| and the
// box-constrained projected-gradient update rho <- clip(rho - alpha G / max|G|, 0, 1)
// (box constraint 0 <= rho <= 1 of Sec. "Methodology", after Eq. 1).
#include <stdint.h>

#include "internal.h"

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
  float m = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(G[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(gmax, __float_as_uint(m));
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

int grid_for(long long n, int per) {
  long long b = (n + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 152 * 8) b = 152 * 8;
  return (int)b;
}

}  // namespace

int launch_j_finalize(const double* part, int n, double* J, cudaStream_t s) {
  k_j_finalize<<<1, 256, 0, s>>>(part, n, J);
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
