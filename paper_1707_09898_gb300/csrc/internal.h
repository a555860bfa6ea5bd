// Internal declarations shared by the translation units of libtopomag.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tmk {

// Lengths the kernels are instantiated for (even 2^a 3^b, b <= 2).
#define TM_FOR_EACH_L(X) \
  X(8) X(12) X(16) X(18) X(24) X(32) X(36) X(48) X(64) X(72) X(96) X(128) X(144) X(192) X(256) X(288) X(384) X(512) X(576)
constexpr int kMaxL = 576;
constexpr int kNT = 256;  // threads per block of every FFT pass

enum XSource { SRC_RHO_CONST = 0, SRC_RHO_FIELD = 1, SRC_VECTOR = 2 };
enum XSink { SINK_FIELD = 0, SINK_OBJECTIVE = 1, SINK_CHAIN = 2 };

// Forward x pass: real rows -> half spectra [3][rows][P] (kx < Lx/2+1 valid, rest 0).
struct XFwdArgs {
  int rows, nx, P;
  int src;                  // XSource
  const float* rho;         // [rows][nx]                (RHO_*)
  const float* M0v;         // [3][rows][nx]             (RHO_FIELD)
  long long M0v_cstride;
  float M0c[3];             // constant M0               (RHO_CONST)
  float p;
  const float* vec;         // [3][rows][nx]             (VECTOR)
  long long vec_cstride;
  float2* out;              // [3][rows][P]
  long long out_cstride;
  const float2* tw;         // W_L^m, m < L
};

// Inverse x pass: half spectra -> real rows, then one of three sinks.
struct XInvArgs {
  int rows, nx, P;
  int sink;                 // XSink
  const float2* in;         // [3][rows][P]
  long long in_cstride;
  float* H;                 // [3][rows][nx] (FIELD; optional in OBJECTIVE)
  long long H_cstride;
  // OBJECTIVE: J = sum_mask sum_c w_c (H_c - Ht_c)^2, g = 2 w (H - Ht) on the mask
  const uint8_t* mask;      // [rows][nx]
  const float* Ht;          // [3][rows][nx] or null -> Htc
  long long Ht_cstride;
  float Htc[3], w[3];
  float2* adj_out;          // [3][rows][P], may alias in
  double* Jpart;            // [gridDim.x]
  // CHAIN: G = p rho^(p-1) M0 . (D g)
  const float* rho;         // [rows][nx]
  const float* M0v;         // [3][rows][nx] or null -> M0c
  long long M0v_cstride;
  float M0c[3];
  float p;
  float* G;                 // [rows][nx]
  unsigned int* gmax;       // max |G| as float bits
  const float2* tw;
};

// y pass over [3][planes][points][P] arrays, tiles of 16 kx columns.
struct YArgs {
  const float2* in;
  float2* out;
  int n_in, n_out, nplanes, P;
  long long in_pstride, out_pstride, in_zstride, out_zstride, in_cstride, out_cstride;
  const float2* tw;
};

// z pass: forward z FFT, tensor product, inverse z FFT, in place on [3][z][Ly][P].
struct ZArgs {
  float2* buf;
  long long cstride, zstride;  // between components, between z planes
  int n_in, n_out, Ly, P;
  const float* T;              // [6][Lz/2+1][Ly/2+1][P]
  long long Tc;                // elements per tensor component
  long long Tz;                // (Ly/2+1) * P
  const int2* zcol;            // launch order of columns: (ky position, ky)
  const float2* tw;
};

int launch_xfwd(int L, const XFwdArgs& a, cudaStream_t s);
int launch_xinv(int L, const XInvArgs& a, cudaStream_t s);
int launch_yfwd(int L, const YArgs& a, cudaStream_t s);
int launch_yinv(int L, const YArgs& a, cudaStream_t s);
int launch_zpass(int L, const ZArgs& a, cudaStream_t s);
int xinv_rows_per_block();
size_t zpass_smem(int L);

// Tensor setup (float64) -- tensor.cu
int tensor_setup(int nx, int ny, int nz, const double d[3], int Lx, int Ly, int Lz, int P, float* T_out,
                 double* octant_host /* optional [6][nz][ny][nx] */, cudaStream_t s, char* err, int errlen);

// Small kernels -- misc.cu
int launch_j_finalize(const double* part, int n, double* J, cudaStream_t s);
int launch_absmax(const float* G, long long n, unsigned int* gmax, cudaStream_t s);
int launch_update(float* rho, const float* G, long long n, float alpha, int normalize, const unsigned int* gmax,
                  cudaStream_t s);

// host mirrors of the digit-reversal maps
int host_pos_of_k(int L, int k);
int host_k_of_pos(int L, int pos);

}  // namespace tmk
