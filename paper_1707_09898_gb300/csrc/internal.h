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

// Programmatic dependent launch. A kernel launched with launch_k(..., pdl = true) is
// queued behind the previous kernel in the stream without the usual launch gap: its
// blocks are placed as the previous grid's blocks exit, do the work that needs nothing
// from predecessors (twiddles into shared memory, barrier set-up, copies of constant
// tables) and call pdl_wait() before they read or write anything a predecessor touches.
// pdl_wait() is a no-op for a kernel launched without the attribute. (An explicit early
// trigger, which lets the next grid's blocks take SM resources while this grid still runs,
// measured slower: 3122 against 3318 evals/s without PDL and 3502 with it as here.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

enum XSource { SRC_RHO_POW = 0, SRC_RHO_M0 = 1, SRC_VECTOR = 2 };
enum XSink { SINK_FIELD = 0, SINK_OBJECTIVE = 1, SINK_CHAIN = 2 };

// Spectral workspaces hold up to kSlots components ("slots"), component-major.
constexpr int kSlotsA = 3;
constexpr int kSlotsB = 4;

// Forward x pass: real rows -> half spectra [slot][rows][P] (kx < Lx/2+1 valid, rest 0).
// One block per (32-row tile, component); blockIdx.y indexes comp[] / out_slot[].
struct XFwdArgs {
  int rows, nx, P;
  int src;                  // XSource
  const float* rho;         // [rows][nx]                       (RHO_*)
  float p;
  const float* M0v;         // [3][rows][nx]                    (RHO_M0: rho^p M0_c)
  long long M0v_cstride;
  const float* vec;         // [3][rows][nx]                    (VECTOR)
  long long vec_cstride;
  int comp[3];              // source component per blockIdx.y
  int out_slot[3];
  float2* out;              // [slot][rows][P]
  long long out_cstride;
  const float2* tw;         // W_L^m, m < L
  // pending projected-gradient step (RHO_POW, one slot, when upd_rho is set): rho is first
  // replaced by min(max(rho - step upd_G, 0), 1) in place, step = upd_alpha / max|upd_G|
  // (max read from *upd_gmax; no step when it is 0) or upd_alpha (upd_normalize == 0)
  float* upd_rho;
  const float* upd_G;
  float upd_alpha;
  int upd_normalize;
  const unsigned int* upd_gmax;
  int pdl;                  // launch with programmatic dependent launch
  unsigned* status;         // device word: bit 0 set when a copy wait timed out (L = 512 one-slot pass)
};
// whether launch_xfwd applies a pending step inside the pass for this length and source
bool xfwd_fuses_step(int L, int src, int ncomp);

// Inverse x pass: half spectra -> real rows, then a sink.
//  FIELD:     block (tile, j): H[comp[j]] = row of slot in_slot[j]
//  OBJECTIVE: block (tile, j): H_c of slot in_slot[j], c = comp[j]; if w_c != 0:
//             J partial, g_c = 2 w_c (H_c - Ht_c) on the mask, forward x transform
//             of g_c written back into slot in_slot[j]
//  CHAIN:     block (tile): G = p rho^(p-1) sum_j coef_j D_j over ncomp slots, where
//             coef_j = M0v[comp[j]] (varying M0) or 1 (slot already contracted with M0)
struct XInvArgs {
  int rows, nx, P;
  int sink;                 // XSink
  int ncomp;
  int comp[3], in_slot[3];
  const float2* in;         // [slot][rows][P]
  long long in_cstride;
  float* H;                 // [3][rows][nx] (FIELD; optional in OBJECTIVE)
  long long H_cstride;
  const uint8_t* mask;      // [rows][nx]
  const float* Ht;          // [3][rows][nx] or null -> Htc
  long long Ht_cstride;
  float Htc[3], w[3];
  float2* adj_out;          // [slot][rows][P], aliases in
  double* Jpart;            // [3][gridDim.x]
  unsigned int* Jcount;     // OBJECTIVE, optional: blocks done; the last one sums Jpart into *Jout
  double* Jout;
  const float* rho;         // [rows][nx]
  const float* M0v;         // [3][rows][nx] or null (contracted slot)
  long long M0v_cstride;
  float p;
  float* G;                 // [rows][nx]
  unsigned int* gmax;       // max |G| as float bits
  const int* ext;           // OBJECTIVE: device [zlo, zhi); blocks outside rows [zlo*ny, zhi*ny) skip
  int ny;
  int row_base;             // first row of block 0 (host-known); rows < `rows` are valid
  const float2* tw;
  int pdl;                  // launch with programmatic dependent launch
  unsigned* status;         // device word: bit 0 set when a copy wait timed out (CHAIN, L = 512)
};

// y pass over [slot][planes][points][P] arrays, tiles of 16 kx columns; blockIdx.z -> in_slot[], out_slot[].
struct YArgs {
  const float2* in;
  float2* out;
  int n_in, n_out, nplanes, P;
  long long in_pstride, out_pstride, in_zstride, out_zstride, in_cstride, out_cstride;
  int in_slot[4], out_slot[4];
  int z0;                   // first plane (host-known offset); planes z0 .. z0 + nplanes - 1
  const int* ext;           // device [zlo, zhi): process only those planes (null: all nplanes)
  const float2* tw;
  int pdl;                  // launch with programmatic dependent launch
};

// z pass, in place on B[slot][z][Ly][P]: forward z transform of nin input slots,
// out_o(k) = sum_i s_oi(k) in_i(k) with s_oi = sum_c coef[o][i][c] N^_c(k) over the six
// unique tensor components (xx, yy, zz, xy, xz, yz), inverse z transform into out_slot[o].
// nin == 1: one block per (tile, column, output). nin > 1: a cluster of nin blocks per
// (tile, column); block r transforms input r and computes output r (r < nout).
struct ZArgs {
  float2* buf;
  long long cstride, zstride;  // between slots, between z planes
  int n_in, n_out, Ly, P;      // input / output z planes
  int nin, nout;
  int in_slot[3], out_slot[3];
  float coef[3][3][6];
  int need[3];                 // per output: bit c set if tensor component c is used
  const float* T;              // [6][Lz/2+1][Ly/2+1][P]
  long long Tc;                // elements per tensor component
  long long Tz;                // (Ly/2+1) * P
  const int2* zcol;            // launch order of columns: (ky position, ky)
  const int* ext;              // device [zlo, zhi) of the target planes
  int in_ext, out_ext;         // input / output planes restricted to ext (else 0..n_in / 0..n_out)
  const float2* tw;
};
constexpr int kDirectPlanes = 4;  // at most this many planes: direct DFT instead of the z FFT

// Direct z convolution (few planes on one side), in place on B[slot][z][Ly][P].
constexpr int kDirectPlanesMax = 8;
struct ZDirArgs {
  float2* buf;
  long long cstride, zstride;
  int P, Ly;
  int nin, nout, in_slot[3], out_slot[3];
  float coef[3][3][6];
  int need[3][3];
  const float* Tz;        // [6][nz][Ly/2+1][P], x/y transformed, z offset
  long long Tc, Tdz;      // per component, per offset
  const int2* zcol;
  int zin0, nzin, zout0, nzout;
};
int launch_zdir(const ZDirArgs& a, cudaStream_t s);

// Fused y transform + direct z sum (k_yzfused.cu).
// Adjoint: from few source planes of B to the real-y rows of every output plane of A.
struct ZYArgs {
  const float2* src;                        // B [slot][z][Ly][P]
  long long src_cstride, src_zstride;
  float2* out;                              // A [slot][z][ny][P]
  long long out_cstride, out_zstride;
  int P, n_out;                             // kx columns (multiple of TB); valid y rows
  int nin, nout, in_slot[3], out_slot[3];
  float coef[3][3][6];
  int need[3][3];
  const float* Tz;                          // [6][nz][Ly/2+1][P]
  long long Tc, Tdz;
  int zin0, nzin, zout0, nzout;
  const float2* tw;                         // W_Ly
  // warp-specialized path (one tensor component c): Ts = coef[0][0][c] * Tz[c], [nzin_total][Ly/2+1][P]
  const float* Ts;
  int nzin_total;                           // z offsets held by Ts
  // if set (warp-specialized path only): the source plane as x spectra, rows [n_src][P]; the
  // kernel runs its forward y transform itself and src is not read
  const float2* gsrc;
  int n_src;
  unsigned* status;                         // device word: bit 0 set when a copy wait timed out
  unsigned* zero_word;                      // if set, zeroed by the warp-specialized kernel (launch_zy_adj returns 1)
  int pdl;                                  // launch with programmatic dependent launch
};
// Forward: the design planes of A onto one plane and one output of B.
struct YZArgs {
  const float2* in;                         // A [slot][z][ny][P]
  long long in_cstride, in_zstride;
  float2* out;                              // B [slot][z][Ly][P]
  long long out_cstride;
  int out_slot;
  float2* part;                             // [z chunks][Ly][P]
  int P, n_in;
  int nin, in_slot[3];
  float coef[3][6];                         // s_i = v^T N u_i of the single output
  int need[3];
  const float* Tz;
  long long Tc, Tdz;
  int zin0, nzin, zchunk, zout;
  const float2* tw;
  // single-component path on two-stage plans (when set): per-block segment partials
  // [2 * blocks][Ly][TB], the target plane's rows in A [ny][P], and the tensor component
  // scaled by its coefficient, Ts = coef[0][c] * Tz[c] [nz_total][Ly/2+1][P]; launch_yz_fwd
  // then also writes the inverse y transform of the target plane there and returns 1
  float2* seg;
  float2* yrows;
  const float* Ts;
  int nz_total;
  unsigned* status;                         // device word: bit 0 set when a copy wait timed out
  int pdl;                                  // launch with programmatic dependent launch
};
int launch_zy_adj(int L, const ZYArgs& a, cudaStream_t s);
// whether launch_zy_adj takes the warp-specialized path for length L (one source plane, one
// spectrum and tensor component, Ts given), the path that can run the source's y transform
bool zy_adj_ws_length(int L);
int launch_yz_fwd(int L, const YZArgs& a, cudaStream_t s);
// after launch_yz_fwd returned 1: the segment partials of each column block added in block
// order, and the target plane's inverse y transform into a.yrows
int launch_yz_finish(int L, const YZArgs& a, cudaStream_t s);

int launch_xfwd(int L, const XFwdArgs& a, int ncomp, cudaStream_t s);
int launch_xinv(int L, const XInvArgs& a, cudaStream_t s);
int launch_yfwd(int L, const YArgs& a, int ncomp, cudaStream_t s);
int launch_yinv(int L, const YArgs& a, int ncomp, cudaStream_t s);
int launch_zpass(int L, const ZArgs& a, cudaStream_t s);
int xinv_rows_per_block();
// Objective on few target rows, compact warp-per-row-pair transforms (k_xobj.cu);
// needs a.Jcount / a.Jout (J summed by the last block) and a.adj_out.
int launch_xobj(int L, const XInvArgs& a, cudaStream_t s);
int xobj_rows_per_block();
size_t zpass_smem(int L);

// Tensor setup (float64) -- tensor.cu
int tensor_setup(int nx, int ny, int nz, const double d[3], int Lx, int Ly, int Lz, int P, float* T_out,
                 float* Tz_out /* optional [6][nz][Ly/2+1][P] */, double* octant_host /* optional [6][nz][ny][nx] */,
                 cudaStream_t s, char* err, int errlen);

// Small kernels -- misc.cu
int launch_j_finalize(const double* part, int n, double* J, cudaStream_t s);
int launch_absmax(const float* G, long long n, unsigned int* gmax, cudaStream_t s);
int launch_mask_extent(const uint8_t* mask, int nz, long long plane, int* ext, cudaStream_t s);
int launch_update(float* rho, const float* G, long long n, float alpha, int normalize, const unsigned int* gmax,
                  cudaStream_t s);
// dst[i] = coef * src[i] (float32 products)
int launch_scale(float* dst, const float* src, long long n, float coef, cudaStream_t s);

// Validation, per-iteration statistics, wait self-test -- misc.cu
// count of entries that are NaN or outside [0, 1] into *bad (zeroed by the caller)
int launch_check_design(const float* rho, long long n, unsigned long long* bad, cudaStream_t s);
// part [2 * nblk] doubles of scratch, out [2]: sum rho, count of 0.1 < rho < 0.9 (fixed order)
int launch_rho_stats(const float* rho, long long n, double* part, int nblk, double* out, cudaStream_t s);
// one block waits at most `polls` polls on an mbarrier phase nothing completes; sets bit 0 of *status
int launch_wait_selftest(unsigned* status, int polls, cudaStream_t s);

// Quadratic stencil objective -- misc.cu
struct StencilArgs {
  long long K, U;                                 // rows, distinct referenced values
  const long long* rp;                            // [K+1] row pointers into idx, a
  const long long* idx;                           // value index into H / gH ([3][nz][ny][nx] flattened)
  const double *a, *c;                            // entry coefficients, row weights [K]
  const long long *cp, *cidx;                     // column form: [U+1] pointers, [U] value indices
  const int* crow;                                // row of each column entry
  const double* ca;                               // coefficient of each column entry
  const float* H;
  float* gH;
  double *r, *part, *J;                           // [K] row values, [nblk] partials, J
  int nblk;
};
int launch_stencil(const StencilArgs& a, cudaStream_t s);

// host mirrors of the digit-reversal maps
int host_pos_of_k(int L, int k);
int host_k_of_pos(int L, int pos);

}  // namespace tmk
