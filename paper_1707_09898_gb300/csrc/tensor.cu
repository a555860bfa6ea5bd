// Demagnetization tensor setup in float64 on the GPU (Sec. "Discretization",
// Eq. (demag_tensor)); run once per grid and excluded from timings, like the
// paper's setup (Sec. "Validation and Benchmarks", Table I caption).
//
// 1. N(R) at every offset R of the non-negative octant [0,nx) x [0,ny) x [0,nz)
//    of the output grid: for max(|i|,|j|,|k|) <= 16 the exact closed form of
//    Newell, Williams and Dunlop (1993) (27-point second differences of f and
//    g with weights -1, 2, -1 per axis); beyond, the cell-cell average of the
//    point-dipole kernel by a 3-node rule per axis on the triangular
//    distribution of the centre separation (nodes 0, +-sqrt(2/5) d; weights
//    7/12, 5/24, exact for its moments up to order 5).
// 2. The transform of the zero-padded, L-periodic tensor. Every component is
//    even or odd along each axis, so its DFT is real and separable into one
//    cosine (even) or sine (odd) sum per axis over the octant; the three sums
//    are evaluated as direct float64 trigonometric sums with an exactly
//    tabulated cos/sin table. Odd axes contribute a factor -i each, so the
//    off-diagonal components (two odd axes) carry a factor -1.
// 3. Scaling by -1/(Lx Ly Lz) (the minus of H = -N*M and the normalisation of
//    the unnormalised inverse transforms), rounding to float32 and storage as
//    [6][Lz/2+1][Ly/2+1][P] with kx padded to P by zeros.
// 4. The same tensor transformed along x and y only (z kept as the offset
//    0 <= dz < nz), scaled by -1/(Lx Ly), float32 [6][nz][Ly/2+1][P]: the z
//    convolution can then be summed directly when one side of it occupies only
//    a few planes. Components odd along exactly one of x, y (xz, yz) are
//    imaginary there; the stored value r means N~ = -i r for them.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "internal.h"

namespace tmk {

namespace {

constexpr int R_NEAR = 16;

__device__ double newell_f(double x, double y, double z) {
  x = fabs(x);
  y = fabs(y);
  z = fabs(z);
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double out = (2.0 * x2 - y2 - z2) * R / 6.0;
  const double rxz = sqrt(x2 + z2), rxy = sqrt(x2 + y2);
  if (y > 0.0 && rxz > 0.0) out += 0.5 * y * (z2 - x2) * asinh(y / rxz);
  if (z > 0.0 && rxy > 0.0) out += 0.5 * z * (y2 - x2) * asinh(z / rxy);
  if (x > 0.0 && y > 0.0 && z > 0.0) out -= x * y * z * atan(y * z / (x * R));
  return out;
}

__device__ double newell_g(double x, double y, double z) {
  const double sgn = (x < 0.0 ? -1.0 : 1.0) * (y < 0.0 ? -1.0 : 1.0);
  x = fabs(x);
  y = fabs(y);
  z = fabs(z);
  if (x == 0.0 || y == 0.0) return 0.0;
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double out = -x * y * R / 3.0;
  out += x * y * z * asinh(z / sqrt(x2 + y2));
  out += y / 6.0 * (3.0 * z2 - y2) * asinh(x / sqrt(y2 + z2));
  out += x / 6.0 * (3.0 * z2 - x2) * asinh(y / sqrt(x2 + z2));
  if (z > 0.0) {
    out -= z2 * z / 6.0 * atan(x * y / (z * R));
    out -= z * y2 / 2.0 * atan(x * z / (y * R));
    out -= z * x2 / 2.0 * atan(y * z / (x * R));
  }
  return sgn * out;
}

__device__ __forceinline__ double sdw(int e) { return e == 0 ? 2.0 : -1.0; }

template <bool G>
__device__ double second_difference(double a, double b, double c, double da, double db, double dc) {
  double acc = 0.0;
  for (int ea = -1; ea <= 1; ea++)
    for (int eb = -1; eb <= 1; eb++)
      for (int ec = -1; ec <= 1; ec++) {
        const double w = sdw(ea) * sdw(eb) * sdw(ec);
        const double x = a + ea * da, y = b + eb * db, z = c + ec * dc;
        acc += w * (G ? newell_g(x, y, z) : newell_f(x, y, z));
      }
  return acc;
}

__device__ void near6(double X, double Y, double Z, double dx, double dy, double dz, double* o) {
  const double k = 1.0 / (4.0 * M_PI * dx * dy * dz);
  o[0] = k * second_difference<false>(X, Y, Z, dx, dy, dz);
  o[1] = k * second_difference<false>(Y, X, Z, dy, dx, dz);
  o[2] = k * second_difference<false>(Z, Y, X, dz, dy, dx);
  o[3] = k * second_difference<true>(X, Y, Z, dx, dy, dz);
  o[4] = k * second_difference<true>(X, Z, Y, dx, dz, dy);
  o[5] = k * second_difference<true>(Y, Z, X, dy, dz, dx);
}

__device__ void far6(double X, double Y, double Z, double dx, double dy, double dz, double* o) {
  const double node = sqrt(0.4);
  const double wts[3] = {5.0 / 24.0, 7.0 / 12.0, 5.0 / 24.0};
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++)
      for (int c = 0; c < 3; c++) {
        const double x = X + (a - 1) * node * dx, y = Y + (b - 1) * node * dy, z = Z + (c - 1) * node * dz;
        const double r2 = x * x + y * y + z * z;
        const double r = sqrt(r2);
        const double i3 = 1.0 / (r2 * r);
        const double i5 = 3.0 * i3 / r2;
        const double w = wts[a] * wts[b] * wts[c];
        acc[0] += w * (i3 - i5 * x * x);
        acc[1] += w * (i3 - i5 * y * y);
        acc[2] += w * (i3 - i5 * z * z);
        acc[3] += w * (-i5 * x * y);
        acc[4] += w * (-i5 * x * z);
        acc[5] += w * (-i5 * y * z);
      }
  const double s = dx * dy * dz / (4.0 * M_PI);
  for (int i = 0; i < 6; i++) o[i] = s * acc[i];
}

// N at offsets (x, y, z) in [0,nx) x [0,ny) x [0,nz): out[6][nz][ny][nx]
__global__ void k_octant(double* out, int nx, int ny, int nz, double dx, double dy, double dz) {
  const long long n = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
    double o[6];
    const int m = max(x, max(y, z));
    if (m <= R_NEAR)
      near6(x * dx, y * dy, z * dz, dx, dy, dz, o);
    else
      far6(x * dx, y * dy, z * dz, dx, dy, dz, o);
    for (int c = 0; c < 6; c++) out[c * n + i] = o[c];
  }
}

// parity bit per component (xx, yy, zz, xy, xz, yz) along x, y, z
constexpr int kOddX = (1 << 3) | (1 << 4);
constexpr int kOddY = (1 << 3) | (1 << 5);
constexpr int kOddZ = (1 << 4) | (1 << 5);

// Transform along the contiguous axis: in[c][line][t] (t < n) -> out[c][line][k] (k < K)
//   out = sum_t w(t) in[t] trig(2 pi k t / L); even: w(0)=1, w(t>0)=2, cos; odd: w(0)=0, w(t>0)=2, sin.
__global__ void k_trig_contig(const double* in, double* out, int lines, int n, int K, int L, int odd_mask,
                              const double* cosT, const double* sinT) {
  extern __shared__ double sh[];
  double* sc = sh;
  double* ss = sh + L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    sc[i] = cosT[i];
    ss[i] = sinT[i];
  }
  __syncthreads();
  const int c = blockIdx.y;
  const bool odd = (odd_mask >> c) & 1;
  const double* tab = odd ? ss : sc;
  const long long total = (long long)lines * K;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
    const long long line = o / K;
    const int k = (int)(o % K);
    const double* row = in + ((long long)c * lines + line) * n;
    double acc = odd ? 0.0 : row[0];
    int idx = k;
    for (int t = 1; t < n; t++) {
      acc += 2.0 * row[t] * tab[idx];
      idx += k;
      if (idx >= L) idx -= L;
    }
    out[((long long)c * lines + line) * K + k] = acc;
  }
}

// Transform along a strided axis: in[c][o][t][i] (t < n) -> out[c][o][k][i] (k < K), i < ni contiguous.
__global__ void k_trig_strided(const double* in, double* out, int outer, int n, int K, int ni, int L, int odd_mask,
                               const double* cosT, const double* sinT) {
  extern __shared__ double sh[];
  double* sc = sh;
  double* ss = sh + L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    sc[i] = cosT[i];
    ss[i] = sinT[i];
  }
  __syncthreads();
  const int c = blockIdx.z / outer, ob = blockIdx.z % outer;
  const int k = blockIdx.y;
  const bool odd = (odd_mask >> c) & 1;
  const double* tab = odd ? ss : sc;
  const double* src = in + ((long long)c * outer + ob) * n * (long long)ni;
  double* dst = out + ((long long)c * outer + ob) * K * (long long)ni;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += gridDim.x * blockDim.x) {
    double acc = odd ? 0.0 : src[i];
    int idx = k;
    for (int t = 1; t < n; t++) {
      acc += 2.0 * src[(long long)t * ni + i] * tab[idx];
      idx += k;
      if (idx >= L) idx -= L;
    }
    dst[(long long)k * ni + i] = acc;
  }
}

// spec[6][KZ][KY][KX] (float64) -> T[6][KZ][KY][P] (float32), scaled; component c
// multiplied by sgn[c] (the product of the -i factors of its odd axes, real part)
__global__ void k_pack(const double* spec, float* T, int KZ, int KY, int KX, int P, double scale, int neg_mask) {
  const long long n = 6LL * KZ * KY * P;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i % P);
    const long long r = i / P;  // (c, kz, ky)
    const int c = (int)(r / ((long long)KZ * KY));
    float v = 0.0f;
    if (k < KX) {
      const double sgn = ((neg_mask >> c) & 1) ? -1.0 : 1.0;
      v = (float)(sgn * scale * spec[r * KX + k]);
    }
    T[i] = v;
  }
}

#define TCK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      snprintf(err, errlen, "tensor setup: %s: %s", #call, cudaGetErrorString(e_));          \
      rc = -1;                                                                               \
      goto done;                                                                             \
    }                                                                                        \
  } while (0)

}  // namespace

int tensor_setup(int nx, int ny, int nz, const double d_in[3], int Lx, int Ly, int Lz, int P, float* T_out,
                 float* Tz_out, double* octant_host, cudaStream_t s, char* err, int errlen) {
  int rc = 0;
  double dmax = fmax(d_in[0], fmax(d_in[1], d_in[2]));
  const double d[3] = {d_in[0] / dmax, d_in[1] / dmax, d_in[2] / dmax};
  const int KX = Lx / 2 + 1, KY = Ly / 2 + 1, KZ = Lz / 2 + 1;
  const long long noct = (long long)nx * ny * nz;
  const long long n1 = (long long)nz * ny * KX, n2 = (long long)nz * KY * KX, n3 = (long long)KZ * KY * KX;
  double *oct = nullptr, *b1 = nullptr, *b2 = nullptr, *tabs = nullptr;
  std::vector<double> htab;
  const int Ls[3] = {Lx, Ly, Lz};
  long long toff[3];

  TCK(cudaMalloc(&oct, 6 * noct * sizeof(double)));
  k_octant<<<(int)((noct + 255) / 256 < 4096 ? (noct + 255) / 256 : 4096), 256, 0, s>>>(oct, nx, ny, nz, d[0], d[1], d[2]);
  TCK(cudaPeekAtLastError());
  if (octant_host) {
    TCK(cudaMemcpyAsync(octant_host, oct, 6 * noct * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  // exact cos/sin tables of 2 pi m / L per axis (host float64)
  {
    long long tot = 0;
    for (int a = 0; a < 3; a++) {
      toff[a] = tot;
      tot += 2LL * Ls[a];
    }
    htab.resize(tot);
    for (int a = 0; a < 3; a++)
      for (int m = 0; m < Ls[a]; m++) {
        htab[toff[a] + m] = cos(2.0 * M_PI * (double)m / (double)Ls[a]);
        htab[toff[a] + Ls[a] + m] = sin(2.0 * M_PI * (double)m / (double)Ls[a]);
      }
    TCK(cudaMalloc(&tabs, tot * sizeof(double)));
    TCK(cudaMemcpyAsync(tabs, htab.data(), tot * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  // x: oct[6][nz*ny][nx] -> b1[6][nz*ny][KX]
  TCK(cudaMalloc(&b1, 6 * n1 * sizeof(double)));
  {
    const long long total = (long long)nz * ny * KX;
    dim3 grid((unsigned)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535), 6);
    k_trig_contig<<<grid, 256, 2 * Lx * sizeof(double), s>>>(oct, b1, nz * ny, nx, KX, Lx, kOddX, tabs + toff[0],
                                                             tabs + toff[0] + Lx);
    TCK(cudaPeekAtLastError());
  }
  TCK(cudaStreamSynchronize(s));
  cudaFree(oct);
  oct = nullptr;
  // y: b1[6][nz][ny][KX] -> b2[6][nz][KY][KX]
  TCK(cudaMalloc(&b2, 6 * n2 * sizeof(double)));
  {
    dim3 grid((KX + 127) / 128, KY, 6 * nz);
    k_trig_strided<<<grid, 128, 2 * Ly * sizeof(double), s>>>(b1, b2, nz, ny, KY, KX, Ly, kOddY, tabs + toff[1],
                                                              tabs + toff[1] + Ly);
    TCK(cudaPeekAtLastError());
  }
  TCK(cudaStreamSynchronize(s));
  cudaFree(b1);
  b1 = nullptr;
  if (Tz_out) {  // x, y transformed; z as offset: xy carries (-i)^2 = -1, xz and yz one -i (kept implicit)
    const long long n = 6LL * nz * KY * P;
    k_pack<<<(int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192), 256, 0, s>>>(
        b2, Tz_out, nz, KY, KX, P, -1.0 / ((double)Lx * (double)Ly), 1 << 3);
    TCK(cudaPeekAtLastError());
  }
  // z: b2[6][1][nz][KY*KX] -> b3[6][KZ][KY*KX]
  TCK(cudaMalloc(&b1, 6 * n3 * sizeof(double)));
  {
    const int ni = KY * KX;
    dim3 grid((ni + 255) / 256 < 64 ? (ni + 255) / 256 : 64, KZ, 6);
    k_trig_strided<<<grid, 256, 2 * Lz * sizeof(double), s>>>(b2, b1, 1, nz, KZ, ni, Lz, kOddZ, tabs + toff[2],
                                                              tabs + toff[2] + Lz);
    TCK(cudaPeekAtLastError());
  }
  {
    const long long n = 6LL * KZ * KY * P;
    k_pack<<<(int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192), 256, 0, s>>>(
        b1, T_out, KZ, KY, KX, P, -1.0 / ((double)Lx * (double)Ly * (double)Lz), (1 << 3) | (1 << 4) | (1 << 5));
    TCK(cudaPeekAtLastError());
  }
  TCK(cudaStreamSynchronize(s));
done:
  if (oct) cudaFree(oct);
  if (b1) cudaFree(b1);
  if (b2) cudaFree(b2);
  if (tabs) cudaFree(tabs);
  return rc;
}

}  // namespace tmk
