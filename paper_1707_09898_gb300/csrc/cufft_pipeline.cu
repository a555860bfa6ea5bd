// Plain cuFFT version of the stray-field objective and adjoint gradient, kept as
// the comparison baseline for the fused sm_103a pipeline (not on the product
// path; built into its own library, libtopomag_cufft.so).
//
// Same mathematics (Sec. "Discretization", Eq. (convolution); Sec.
// "Methodology", Eqs. (adjoint1)-(adjoint2)), done the textbook way: explicit
// zero padding of rho^p M0 into [3][Lz][Ly][Lx] real arrays, cufftExecR2C
// (3-D, batch 3), the product with the full complex64 tensor
// [6][Lz][Ly][Lx/2+1], cufftExecC2R, crop + least-squares objective + dJ/dH
// into a zero-padded array, and the same again for the adjoint, then the chain
// rule on the design box.
#include <cufft.h>
#include <stdint.h>
#include <stdio.h>

#include <vector>

extern "C" {
typedef struct tmb_ctx tmb_ctx;
int tmb_create(tmb_ctx** out, int device, const int n_out[3], int nzd, const int L[3]);
void tmb_destroy(tmb_ctx* b);
int tmb_set_tensor(tmb_ctx* b, const float* folded_host /* [6][Lz/2+1][Ly/2+1][Lx/2+1], already scaled */);
int tmb_set_M0(tmb_ctx* b, const double M0[3], double p);
int tmb_objective_and_gradient(tmb_ctx* b, const float* rho, const uint8_t* mask, const float Ht_const[3],
                               const float w[3], float* dJdrho, void* stream);
int tmb_get_objective(tmb_ctx* b, double* J, void* stream);
}

struct tmb_ctx {
  int dev, nx, ny, nz, nzd, Lx, Ly, Lz, K;
  long long nr, nc;  // real / complex elements per component
  float* real = nullptr;
  cufftComplex* spec = nullptr;
  cufftComplex* T = nullptr;  // [6][Lz][Ly][K]
  double* Jpart = nullptr;
  double* J = nullptr;
  double Jh = 0;
  float M0[3] = {0, 0, 0};
  float p = 3.0f;
  cufftHandle fwd = 0, inv = 0;
  int nblk = 0;
};

namespace {

__global__ void k_pad_rho(const float* rho, float* real, int nx, int ny, int nzd, int Lx, int Ly, long long nr, float p,
                          float m0x, float m0y, float m0z) {
  const long long n = 3 * nr;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / nr);
    const long long r = i - c * nr;
    const int x = (int)(r % Lx), y = (int)((r / Lx) % Ly), z = (int)(r / ((long long)Lx * Ly));
    float v = 0.0f;
    if (x < nx && y < ny && z < nzd) {
      const float rv = rho[((long long)z * ny + y) * nx + x];
      const float m = c == 0 ? m0x : c == 1 ? m0y : m0z;
      v = powf(rv, p) * m;
    }
    real[i] = v;
  }
}

// H_c = sum_d T_cd M_d (T symmetric, 6 unique components)
__global__ void k_mul(cufftComplex* spec, const cufftComplex* T, long long nc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
    const cufftComplex mx = spec[i], my = spec[nc + i], mz = spec[2 * nc + i];
    const cufftComplex xx = T[i], yy = T[nc + i], zz = T[2 * nc + i], xy = T[3 * nc + i], xz = T[4 * nc + i],
                       yz = T[5 * nc + i];
    auto mul = [](cufftComplex a, cufftComplex b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    auto add3 = [](float2 a, float2 b, float2 c) { return make_float2(a.x + b.x + c.x, a.y + b.y + c.y); };
    spec[i] = add3(mul(xx, mx), mul(xy, my), mul(xz, mz));
    spec[nc + i] = add3(mul(xy, mx), mul(yy, my), mul(yz, mz));
    spec[2 * nc + i] = add3(mul(xz, mx), mul(yz, my), mul(zz, mz));
  }
}

// crop H, objective partials, g = 2 w (H - Ht) on the mask into the (re-zeroed) padded arrays
__global__ void k_objective(float* real, const uint8_t* mask, int nx, int ny, int nz, int Lx, int Ly, long long nr,
                            float h0, float h1, float h2, float w0, float w1, float w2, double* Jpart) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr; r += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(r % Lx), y = (int)((r / Lx) % Ly), z = (int)(r / ((long long)Lx * Ly));
    float g[3] = {0, 0, 0};
    if (x < nx && y < ny && z < nz && mask[((long long)z * ny + y) * nx + x]) {
      const float ht[3] = {h0, h1, h2}, w[3] = {w0, w1, w2};
      for (int c = 0; c < 3; c++) {
        const float d = real[c * nr + r] - ht[c];
        acc += (double)w[c] * d * d;
        g[c] = 2.0f * w[c] * d;
      }
    }
    for (int c = 0; c < 3; c++) real[c * nr + r] = g[c];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) Jpart[blockIdx.x] = red[0];
}

__global__ void k_sum(const double* part, int n, double* J) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += part[i];
    *J = s;
  }
}

__global__ void k_chain(const float* real, const float* rho, float* G, int nx, int ny, int nzd, int Lx, int Ly,
                        long long nr, float p, float m0x, float m0y, float m0z) {
  const long long n = (long long)nx * ny * nzd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    const long long r = ((long long)z * Ly + y) * Lx + x;
    const float d = m0x * real[r] + m0y * real[nr + r] + m0z * real[2 * nr + r];
    G[i] = p * powf(rho[i], p - 1.0f) * d;
  }
}

// unfold the real parity-folded tensor into the full complex64 one
__global__ void k_unfold(const float* F, cufftComplex* T, int Lx, int Ly, int Lz, int K) {
  const int KY = Ly / 2 + 1, KZ = Lz / 2 + 1;
  const long long nc = (long long)Lz * Ly * K;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 6 * nc; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / nc);
    const long long r = i - c * nc;
    const int kx = (int)(r % K), ky = (int)((r / K) % Ly), kz = (int)(r / ((long long)K * Ly));
    const int kyf = ky <= Ly / 2 ? ky : Ly - ky, kzf = kz <= Lz / 2 ? kz : Lz - kz;
    float v = F[(((long long)c * KZ + kzf) * KY + kyf) * K + kx];
    const bool oy = (c == 3 || c == 5), oz = (c == 4 || c == 5);
    if (oy && ky > Ly / 2) v = -v;
    if (oz && kz > Lz / 2) v = -v;
    T[i] = make_float2(v, 0.0f);
  }
}

int grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b > 8192 ? 8192 : (b < 1 ? 1 : b));
}

}  // namespace

extern "C" int tmb_create(tmb_ctx** out, int device, const int n_out[3], int nzd, const int L[3]) {
  if (!out) return -1;
  if (cudaSetDevice(device) != cudaSuccess) return -4;
  tmb_ctx* b = new tmb_ctx();
  b->dev = device;
  b->nx = n_out[0];
  b->ny = n_out[1];
  b->nz = n_out[2];
  b->nzd = nzd;
  b->Lx = L[0];
  b->Ly = L[1];
  b->Lz = L[2];
  b->K = L[0] / 2 + 1;
  b->nr = (long long)L[0] * L[1] * L[2];
  b->nc = (long long)b->K * L[1] * L[2];
  b->nblk = 1024;
  int n[3] = {L[2], L[1], L[0]};
  bool ok = cudaMalloc(&b->real, 3 * b->nr * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&b->spec, 3 * b->nc * sizeof(cufftComplex)) == cudaSuccess &&
            cudaMalloc(&b->T, 6 * b->nc * sizeof(cufftComplex)) == cudaSuccess &&
            cudaMalloc(&b->Jpart, b->nblk * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&b->J, sizeof(double)) == cudaSuccess &&
            cufftPlanMany(&b->fwd, 3, n, nullptr, 1, (int)b->nr, nullptr, 1, (int)b->nc, CUFFT_R2C, 3) ==
                CUFFT_SUCCESS &&
            cufftPlanMany(&b->inv, 3, n, nullptr, 1, (int)b->nc, nullptr, 1, (int)b->nr, CUFFT_C2R, 3) ==
                CUFFT_SUCCESS;
  if (!ok) {
    tmb_destroy(b);
    return -5;
  }
  *out = b;
  return 0;
}

extern "C" void tmb_destroy(tmb_ctx* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  if (b->fwd) cufftDestroy(b->fwd);
  if (b->inv) cufftDestroy(b->inv);
  cudaFree(b->real);
  cudaFree(b->spec);
  cudaFree(b->T);
  cudaFree(b->Jpart);
  cudaFree(b->J);
  delete b;
}

extern "C" int tmb_set_tensor(tmb_ctx* b, const float* folded_host) {
  const size_t n = 6ULL * (b->Lz / 2 + 1) * (b->Ly / 2 + 1) * b->K;
  float* F = nullptr;
  if (cudaMalloc(&F, n * sizeof(float)) != cudaSuccess) return -5;
  cudaMemcpy(F, folded_host, n * sizeof(float), cudaMemcpyHostToDevice);
  k_unfold<<<grid(6 * b->nc), 256>>>(F, b->T, b->Lx, b->Ly, b->Lz, b->K);
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(F);
  return e == cudaSuccess ? 0 : -4;
}

extern "C" int tmb_set_M0(tmb_ctx* b, const double M0[3], double p) {
  for (int c = 0; c < 3; c++) b->M0[c] = (float)M0[c];
  b->p = (float)p;
  return 0;
}

extern "C" int tmb_objective_and_gradient(tmb_ctx* b, const float* rho, const uint8_t* mask, const float Ht_const[3],
                                          const float w[3], float* dJdrho, void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cufftSetStream(b->fwd, s);
  cufftSetStream(b->inv, s);
  k_pad_rho<<<grid(3 * b->nr), 256, 0, s>>>(rho, b->real, b->nx, b->ny, b->nzd, b->Lx, b->Ly, b->nr, b->p, b->M0[0],
                                             b->M0[1], b->M0[2]);
  if (cufftExecR2C(b->fwd, b->real, b->spec) != CUFFT_SUCCESS) return -4;
  k_mul<<<grid(b->nc), 256, 0, s>>>(b->spec, b->T, b->nc);
  if (cufftExecC2R(b->inv, b->spec, b->real) != CUFFT_SUCCESS) return -4;
  k_objective<<<b->nblk, 256, 0, s>>>(b->real, mask, b->nx, b->ny, b->nz, b->Lx, b->Ly, b->nr, Ht_const[0],
                                      Ht_const[1], Ht_const[2], w[0], w[1], w[2], b->Jpart);
  k_sum<<<1, 32, 0, s>>>(b->Jpart, b->nblk, b->J);
  if (cufftExecR2C(b->fwd, b->real, b->spec) != CUFFT_SUCCESS) return -4;
  k_mul<<<grid(b->nc), 256, 0, s>>>(b->spec, b->T, b->nc);
  if (cufftExecC2R(b->inv, b->spec, b->real) != CUFFT_SUCCESS) return -4;
  k_chain<<<grid((long long)b->nx * b->ny * b->nzd), 256, 0, s>>>(b->real, rho, dJdrho, b->nx, b->ny, b->nzd, b->Lx,
                                                                  b->Ly, b->nr, b->p, b->M0[0], b->M0[1], b->M0[2]);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -4;
}

extern "C" int tmb_get_objective(tmb_ctx* b, double* J, void* stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaMemcpyAsync(&b->Jh, b->J, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -4;
  *J = b->Jh;
  return 0;
}
