// C ABI of libtopomag: context, workspace and the pass sequences of the
// stray-field operator D, its adjoint, the fused objective/gradient and the
// projected update. Every array argument is a caller-owned device pointer.
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/topomag.h"
#include "fft.cuh"
#include "internal.h"

using namespace tmk;

struct tm_ctx {
  int device = 0;
  int nx = 0, ny = 0, nz = 0, nzd = 0;
  double d[3] = {0, 0, 0};
  int L[3] = {0, 0, 0};
  int P = 0;
  double p = 3.0;
  bool have_grid = false, have_tensor = false, have_M0 = false;
  bool m0_var = false;
  double M0c[3] = {0, 0, 0};
  float* M0v = nullptr;     // [3][nzd][ny][nx]
  float* T = nullptr;       // [6][Lz/2+1][Ly/2+1][P]
  float* Tz = nullptr;      // [6][nz][Ly/2+1][P] (x, y transformed; z offset)
  // prepared target (tm_set_target)
  bool have_target = false;
  uint8_t* tmask = nullptr;  // [nz][ny][nx]
  float* tHt = nullptr;      // [3][nz][ny][nx] or null
  float tHtc[3] = {0, 0, 0}, tw_[3] = {0, 0, 0};
  int tz0 = 0, tz1 = 0;      // planes holding target cells
  // prepared stencil objective (tm_set_stencil_objective): target_kind 1
  int target_kind = 0;
  long long sK = 0, sU = 0;
  long long *s_rp = nullptr, *s_idx = nullptr, *s_cp = nullptr, *s_cidx = nullptr;
  double *s_a = nullptr, *s_c = nullptr, *s_ca = nullptr, *s_r = nullptr, *s_part = nullptr;
  int* s_crow = nullptr;
  int s_comps = 0;                      // bit c set: component c is referenced
  float *sH = nullptr, *sgH = nullptr;  // [3][nz][ny][nx] field / dJ/dH buffers
  float2* A = nullptr;      // [3][nz][ny][P]
  float2* B = nullptr;      // [4][nz][Ly][P]
  float2* tw = nullptr;     // twiddles: Lx | Ly | Lz
  int2* zcol = nullptr;     // [Ly]
  double* Jpart = nullptr;  // [ceil(nz*ny/rows_per_block)]
  int nJpart = 0;
  double* Jdev = nullptr;
  unsigned int* gmax = nullptr;
  const float* gmax_of = nullptr;  // the array whose max |.| gmax holds (set by the chain-rule pass)
  // projected-gradient step that tm_evaluate_step hands to the x forward pass of rho
  unsigned* dstat = nullptr;       // device status word of the TMA-fed kernels (bit 0: a copy wait timed out)
  unsigned* hstat = nullptr;       // pinned host copy
  bool pdl = true;                 // launch the passes with programmatic dependent launch
  bool gmax_zeroed = false;        // the fused adjoint cleared gmax for the chain-rule pass
  float* pend_rho = nullptr;
  const float* pend_G = nullptr;
  float pend_alpha = 0.0f;
  int pend_normalize = 0;
  unsigned int* Jcount = nullptr;  // blocks of the objective pass done (re-armed by the last one)
  bool fuse_yz = true;             // prepared path: y transform fused with the direct z sum
  float2* yzpart = nullptr;        // [z chunks][Ly][P] partial planes of the fused forward
  int yzpart_chunks = 0;
  float2* yzseg = nullptr;         // [2 * SMs][Ly][TB] segment partials of the flattened fused forward
  // one tensor component times its coupling coefficient, for the fused forward (0) and
  // adjoint (1): [nz][Ly/2+1][P], rebuilt when the component, the coefficient or the tensor change
  float* Ts[2] = {nullptr, nullptr};
  int Ts_comp[2] = {-1, -1};
  float Ts_coef[2] = {0.0f, 0.0f};
  long long Ts_gen[2] = {-1, -1};
  long long tensor_gen = 0;        // counts tm_set_tensor calls
  int nsm = 0;
  int* ext = nullptr;       // [2]: z range of the target planes
  double* stats = nullptr;  // [2 * kStatBlocks + 2] scratch of tm_iteration_stats
  unsigned long long* nbad = nullptr;  // count of tm_check_design
  double* Jhost = nullptr;  // pinned
  // per-kernel event timing (tm_profile)
  bool prof_on = false;
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  char err[512] = {0};
};

namespace {

int fail(tm_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

// Fault injection (tm_inject_fault / TM_FAULT_INJECT=<call>[:<nth>]): the armed call
// fails with TM_ERR_INJECTED on its nth invocation, before it touches any state.
struct Injection {
  std::mutex mu;
  std::string call;
  long long left = 0;
  Injection() {
    const char* e = getenv("TM_FAULT_INJECT");
    if (!e || !*e) return;
    std::string v(e);
    const size_t c = v.find(':');
    call = v.substr(0, c);
    left = c == std::string::npos ? 1 : atoll(v.c_str() + c + 1);
  }
};
Injection& injection() {
  static Injection inj;
  return inj;
}
bool injected(const char* name) {
  Injection& in = injection();
  std::lock_guard<std::mutex> lock(in.mu);
  if (in.left <= 0 || in.call != name) return false;
  if (--in.left > 0) return false;
  in.call.clear();
  return true;
}
// Entry points called from inside another one (tm_evaluate_step -> tm_evaluate) do not
// count: only calls made by the caller of the library do. Each entry point is also an
// NVTX range named after it (free when no profiler is attached).
thread_local int tl_depth = 0;
struct DepthGuard {
  explicit DepthGuard(const char* name) {
    tl_depth++;
    nvtxRangePushA(name);
  }
  ~DepthGuard() {
    nvtxRangePop();
    tl_depth--;
  }
};
#define INJECT(ctx, name)                                                                       \
  if (tl_depth == 0 && injected(name))                                                          \
    return fail(ctx, TM_ERR_INJECTED, "%s: failure injected by tm_inject_fault", name);         \
  DepthGuard depth_guard_(name)

// Reads the device status word (synchronising `s`); a set bit 0 means that a bounded
// wait ran out in some kernel since the word was last cleared.
int check_status(tm_ctx* ctx, cudaStream_t s);

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? TM_ERR_NOMEM : TM_ERR_CUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                         \
  } while (0)

#define CKL(call)                                                                                  \
  do {                                                                                             \
    int r_ = (call);                                                                               \
    if (r_ != 0) {                                                                                 \
      cudaError_t e_ = cudaGetLastError();                                                         \
      return fail(ctx, r_ == -2 ? TM_ERR_SIZE : TM_ERR_CUDA, "%s failed: %s", #call,               \
                  cudaGetErrorString(e_));                                                         \
    }                                                                                              \
  } while (0)

int check_status(tm_ctx* ctx, cudaStream_t s) {
  CK(cudaMemcpyAsync(ctx->hstat, ctx->dstat, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (*ctx->hstat) {
    CK(cudaMemsetAsync(ctx->dstat, 0, sizeof(unsigned), s));
    CK(cudaStreamSynchronize(s));
    return fail(ctx, TM_ERR_TIMEOUT, "a bounded wait for a tensor-memory-accelerator copy ran out in a kernel; "
                                     "the results since the last check are invalid");
  }
  return TM_OK;
}

bool supported_L(int L) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return true;
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return false;
}

// Default padded length of an axis of n cells: the smallest supported L >= 2 n, except that
// a length strictly between 256 and 512 is replaced by 512. Any L >= 2 n gives the same
// linear convolution; 512 = 32 x 16 has the fused and warp-specialized kernels, the
// three-stage lengths 288 and 384 only the general ones (measured at 192^3: 0.246 ms per
// evaluation with L = 384, 0.174 ms with L = 512).
int pick_length(int n) {
  static const int ls[] = {
#define TM_LIST(LL) LL,
      TM_FOR_EACH_L(TM_LIST)
#undef TM_LIST
  };
  for (int L : ls)
    if (L >= 2 * n) return (L > 256 && L < 512) ? 512 : L;
  return 0;
}

void free_stencil(tm_ctx* c) {
  void* ps[] = {c->s_rp, c->s_idx, c->s_cp, c->s_cidx, c->s_a, c->s_c, c->s_ca, c->s_r, c->s_part, c->s_crow};
  for (void* p : ps) cudaFree(p);
  c->s_rp = c->s_idx = c->s_cp = c->s_cidx = nullptr;
  c->s_a = c->s_c = c->s_ca = c->s_r = c->s_part = nullptr;
  c->s_crow = nullptr;
  c->sK = c->sU = 0;
}

void free_grid(tm_ctx* c) {
  free_stencil(c);
  cudaFree(c->yzpart);
  c->yzpart = nullptr;
  c->yzpart_chunks = 0;
  cudaFree(c->yzseg);
  c->yzseg = nullptr;
  for (int k = 0; k < 2; k++) {
    cudaFree(c->Ts[k]);
    c->Ts[k] = nullptr;
    c->Ts_comp[k] = -1;
  }
  cudaFree(c->sH);
  cudaFree(c->sgH);
  c->sH = c->sgH = nullptr;
  c->target_kind = 0;
  cudaFree(c->M0v);
  cudaFree(c->T);
  cudaFree(c->Tz);
  cudaFree(c->tmask);
  cudaFree(c->tHt);
  c->Tz = nullptr;
  c->tmask = nullptr;
  c->tHt = nullptr;
  c->have_target = false;
  cudaFree(c->A);
  cudaFree(c->B);
  cudaFree(c->tw);
  cudaFree(c->zcol);
  cudaFree(c->Jpart);
  c->M0v = nullptr;
  c->T = nullptr;
  c->A = c->B = c->tw = nullptr;
  c->zcol = nullptr;
  c->Jpart = nullptr;
  c->have_grid = c->have_tensor = c->have_M0 = false;
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

enum { KIND_XFWD = 0, KIND_YFWD, KIND_ZPASS, KIND_YINV, KIND_XINV, KIND_OTHER, KIND_YZF, KIND_ZYA, KIND_OBJ, KIND_N };

// Records a start/stop event pair around one launch when profiling is on.
struct Timed {
  tm_ctx* c;
  cudaStream_t s;
  size_t slot = (size_t)-1;
  Timed(tm_ctx* ctx, int kind, cudaStream_t st) : c(ctx), s(st) {
    if (!c->prof_on) return;
    if (c->ev_used * 2 + 2 > c->ev.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return;
      }
      c->ev.push_back(a);
      c->ev.push_back(b);
      c->ev_kind.push_back(kind);
    }
    slot = c->ev_used++;
    c->ev_kind[slot] = kind;
    cudaEventRecord(c->ev[2 * slot], s);
  }
  ~Timed() {
    if (slot != (size_t)-1) cudaEventRecord(c->ev[2 * slot + 1], s);
  }
};

long long design_cells(const tm_ctx* c) { return (long long)c->nzd * c->ny * c->nx; }
long long out_cells(const tm_ctx* c) { return (long long)c->nz * c->ny * c->nx; }

int check_ready(tm_ctx* ctx) {
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  if (!ctx->have_tensor) return fail(ctx, TM_ERR_STATE, "no tensor: call tm_set_tensor first");
  if (!ctx->have_M0) return fail(ctx, TM_ERR_STATE, "no M0: call tm_set_M0 first");
  CK(cudaSetDevice(ctx->device));
  return TM_OK;
}

// coefficients of s = v^T N u over the unique components (xx, yy, zz, xy, xz, yz)
void coef6(float c[6], const double v[3], const double u[3]) {
  c[0] = (float)(v[0] * u[0]);
  c[1] = (float)(v[1] * u[1]);
  c[2] = (float)(v[2] * u[2]);
  c[3] = (float)(v[0] * u[1] + v[1] * u[0]);
  c[4] = (float)(v[0] * u[2] + v[2] * u[0]);
  c[5] = (float)(v[1] * u[2] + v[2] * u[1]);
}
const double kUnit[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

// One application of the y / z / y passes. Inputs: nin spectra in A slots ain[]
// (zin planes); outputs: nout spectra in A slots aout[] (zout planes) with
// out_o = sum_i (v_o^T N u_i) in_i. B slots: inputs go to bin[], outputs to bout[].
struct ConvSpec {
  int nin, nout;
  int ain[3], bin[3], bout[3], aout[3];
  const double* u[3];  // per input
  const double* v[3];  // per output
  const int* ext;      // device z range of the target planes, used when in_ext / out_ext
  int in_ext, out_ext;
};

int conv_yz(tm_ctx* ctx, const ConvSpec& cs, int zin, int zout, cudaStream_t s) {
  const int Lx = ctx->L[0], Ly = ctx->L[1], Lz = ctx->L[2];
  const long long P = ctx->P;
  const long long A_cs = (long long)ctx->nz * ctx->ny * P, B_cs = (long long)ctx->nz * Ly * P;
  YArgs y{};
  y.in = ctx->A;
  y.out = ctx->B;
  y.n_in = ctx->ny;
  y.n_out = Ly;
  y.nplanes = zin;
  y.P = ctx->P;
  y.in_pstride = P;
  y.out_pstride = P;
  y.in_zstride = (long long)ctx->ny * P;
  y.out_zstride = (long long)Ly * P;
  y.in_cstride = A_cs;
  y.out_cstride = B_cs;
  for (int i = 0; i < cs.nin; i++) {
    y.in_slot[i] = cs.ain[i];
    y.out_slot[i] = cs.bin[i];
  }
  y.ext = cs.in_ext ? cs.ext : nullptr;
  y.tw = ctx->tw + Lx;
  {
    Timed t(ctx, KIND_YFWD, s);
    CKL(launch_yfwd(Ly, y, cs.nin, s));
  }

  ZArgs z{};
  z.buf = ctx->B;
  z.cstride = B_cs;
  z.zstride = (long long)Ly * P;
  z.n_in = zin;
  z.n_out = zout;
  z.Ly = Ly;
  z.P = ctx->P;
  z.nin = cs.nin;
  z.nout = cs.nout;
  for (int i = 0; i < cs.nin; i++) z.in_slot[i] = cs.bin[i];
  for (int o = 0; o < cs.nout; o++) {
    z.out_slot[o] = cs.bout[o];
    z.need[o] = 0;
    for (int i = 0; i < cs.nin; i++) {
      coef6(z.coef[o][i], cs.v[o], cs.u[i]);
      for (int c = 0; c < 6; c++)
        if (z.coef[o][i][c] != 0.0f) z.need[o] |= 1 << c;
    }
  }
  z.T = ctx->T;
  z.Tz = (long long)(Ly / 2 + 1) * P;
  z.Tc = (long long)(Lz / 2 + 1) * z.Tz;
  z.zcol = ctx->zcol;
  z.ext = cs.ext;
  z.in_ext = cs.in_ext;
  z.out_ext = cs.out_ext;
  z.tw = ctx->tw + Lx + Ly;
  {
    Timed t(ctx, KIND_ZPASS, s);
    CKL(launch_zpass(Lz, z, s));
  }

  YArgs yi{};
  yi.in = ctx->B;
  yi.out = ctx->A;
  yi.n_in = Ly;
  yi.n_out = ctx->ny;
  yi.nplanes = zout;
  yi.P = ctx->P;
  yi.in_pstride = P;
  yi.out_pstride = P;
  yi.in_zstride = (long long)Ly * P;
  yi.out_zstride = (long long)ctx->ny * P;
  yi.in_cstride = B_cs;
  yi.out_cstride = A_cs;
  for (int o = 0; o < cs.nout; o++) {
    yi.in_slot[o] = cs.bout[o];
    yi.out_slot[o] = cs.aout[o];
  }
  yi.ext = cs.out_ext ? cs.ext : nullptr;
  yi.tw = ctx->tw + Lx;
  {
    Timed t(ctx, KIND_YINV, s);
    CKL(launch_yinv(Ly, yi, cs.nout, s));
  }
  return TM_OK;
}

// y pass (forward or inverse) over planes [z0, z0 + np) between A slots and B slots
int ypass(tm_ctx* ctx, bool inv, int n, const int* aslot, const int* bslot, int z0, int np, cudaStream_t s) {
  const int Lx = ctx->L[0], Ly = ctx->L[1];
  const long long P = ctx->P;
  YArgs y{};
  y.in = inv ? ctx->B : ctx->A;
  y.out = inv ? ctx->A : ctx->B;
  y.n_in = inv ? Ly : ctx->ny;
  y.n_out = inv ? ctx->ny : Ly;
  y.nplanes = np;
  y.P = ctx->P;
  y.in_pstride = P;
  y.out_pstride = P;
  y.in_zstride = (inv ? (long long)Ly : (long long)ctx->ny) * P;
  y.out_zstride = (inv ? (long long)ctx->ny : (long long)Ly) * P;
  y.in_cstride = inv ? (long long)ctx->nz * Ly * P : (long long)ctx->nz * ctx->ny * P;
  y.out_cstride = inv ? (long long)ctx->nz * ctx->ny * P : (long long)ctx->nz * Ly * P;
  for (int i = 0; i < n; i++) {
    y.in_slot[i] = inv ? bslot[i] : aslot[i];
    y.out_slot[i] = inv ? aslot[i] : bslot[i];
  }
  y.z0 = z0;
  y.tw = ctx->tw + Lx;
  y.pdl = ctx->pdl;
  Timed t(ctx, inv ? KIND_YINV : KIND_YFWD, s);
  CKL(inv ? launch_yinv(Ly, y, n, s) : launch_yfwd(Ly, y, n, s));
  return TM_OK;
}

// direct z convolution between B slots: inputs planes [zi0, zi0 + nzi), outputs [zo0, zo0 + nzo)
int zdirect(tm_ctx* ctx, const ConvSpec& cs, int zi0, int nzi, int zo0, int nzo, cudaStream_t s) {
  const int Ly = ctx->L[1];
  const long long P = ctx->P;
  ZDirArgs z{};
  z.buf = ctx->B;
  z.cstride = (long long)ctx->nz * Ly * P;
  z.zstride = (long long)Ly * P;
  z.P = ctx->P;
  z.Ly = Ly;
  z.nin = cs.nin;
  z.nout = cs.nout;
  for (int i = 0; i < cs.nin; i++) z.in_slot[i] = cs.bin[i];
  for (int o = 0; o < cs.nout; o++) {
    z.out_slot[o] = cs.bout[o];
    for (int i = 0; i < cs.nin; i++) {
      coef6(z.coef[o][i], cs.v[o], cs.u[i]);
      z.need[o][i] = 0;
      for (int c = 0; c < 6; c++)
        if (z.coef[o][i][c] != 0.0f) z.need[o][i] |= 1 << c;
    }
  }
  z.Tz = ctx->Tz;
  z.Tdz = (long long)(Ly / 2 + 1) * P;
  z.Tc = (long long)ctx->nz * z.Tdz;
  z.zcol = ctx->zcol;
  z.zin0 = zi0;
  z.nzin = nzi;
  z.zout0 = zo0;
  z.nzout = nzo;
  Timed t(ctx, KIND_ZPASS, s);
  CKL(launch_zdir(z, s));
  return TM_OK;
}

// Tensor component c times coef, [nz][Ly/2+1][P], for the fused kernel `which` (0 forward,
// 1 adjoint); kept until the component, the coefficient or the tensor change. *rebuilt:
// it was (re)computed on the stream just now, so the next launch must not overlap it.
int scaled_component(tm_ctx* ctx, int which, int c, float coef, cudaStream_t s, const float** out, bool* rebuilt) {
  *rebuilt = false;
  const long long n = (long long)ctx->nz * (ctx->L[1] / 2 + 1) * ctx->P;
  if (!ctx->Ts[which]) CK(cudaMalloc(&ctx->Ts[which], n * sizeof(float)));
  if (ctx->Ts_comp[which] != c || ctx->Ts_coef[which] != coef || ctx->Ts_gen[which] != ctx->tensor_gen) {
    CKL(launch_scale(ctx->Ts[which], ctx->Tz + c * n, n, coef, s));
    *rebuilt = true;
    ctx->Ts_comp[which] = c;
    ctx->Ts_coef[which] = coef;
    ctx->Ts_gen[which] = ctx->tensor_gen;
  }
  *out = ctx->Ts[which];
  return TM_OK;
}

int one_component(int need) { return (need != 0 && (need & (need - 1)) == 0) ? __builtin_ctz(need) : -1; }

// forward y transform of the design planes fused with the direct z sum onto the
// single target plane (cs.nout == 1); *yinv_done: the kernel also wrote the target
// plane's inverse y transform into A
int yz_forward(tm_ctx* ctx, const ConvSpec& cs, int zo, cudaStream_t s, bool* yinv_done) {
  const int Ly = ctx->L[1];
  const long long P = ctx->P;
  const int chunks = (int)(P / TB);
  int nch = ctx->nsm / chunks;  // one resident block per SM: a single wave
  nch = nch < 1 ? 1 : (nch > ctx->nzd ? ctx->nzd : nch);
  const int zchunk = (ctx->nzd + nch - 1) / nch;
  nch = (ctx->nzd + zchunk - 1) / zchunk;
  if (nch > ctx->yzpart_chunks) {
    cudaFree(ctx->yzpart);
    ctx->yzpart = nullptr;
    ctx->yzpart_chunks = 0;
    CK(cudaMalloc(&ctx->yzpart, (size_t)nch * Ly * P * sizeof(float2)));
    ctx->yzpart_chunks = nch;
  }
  YZArgs y{};
  y.in = ctx->A;
  y.in_cstride = (long long)ctx->nz * ctx->ny * P;
  y.in_zstride = (long long)ctx->ny * P;
  y.out = ctx->B;
  y.out_cstride = (long long)ctx->nz * Ly * P;
  y.out_slot = cs.bout[0];
  y.part = ctx->yzpart;
  y.P = ctx->P;
  y.n_in = ctx->ny;
  y.nin = cs.nin;
  for (int i = 0; i < cs.nin; i++) {
    y.in_slot[i] = cs.ain[i];
    coef6(y.coef[i], cs.v[0], cs.u[i]);
    y.need[i] = 0;
    for (int c = 0; c < 6; c++)
      if (y.coef[i][c] != 0.0f) y.need[i] |= 1 << c;
  }
  y.Tz = ctx->Tz;
  y.Tdz = (long long)(Ly / 2 + 1) * P;
  y.Tc = (long long)ctx->nz * y.Tdz;
  y.zin0 = 0;
  y.nzin = ctx->nzd;
  y.zchunk = zchunk;
  y.zout = zo;
  y.tw = ctx->tw + ctx->L[0];
  if (!ctx->yzseg) CK(cudaMalloc(&ctx->yzseg, (size_t)2 * ctx->nsm * Ly * TB * sizeof(float2)));
  y.seg = ctx->yzseg;
  const int c1 = cs.nin == 1 ? one_component(y.need[0]) : -1;
  if (c1 >= 0) {
    int r;
    bool rebuilt;
    if ((r = scaled_component(ctx, 0, c1, y.coef[0][c1], s, &y.Ts, &rebuilt))) return r;
    y.nz_total = ctx->nz;
  }
  y.status = ctx->dstat;
  y.yrows = ctx->A + cs.aout[0] * ((long long)ctx->nz * ctx->ny * P) + (long long)zo * ctx->ny * P;
  y.pdl = ctx->pdl;
  int r;
  {
    Timed t(ctx, KIND_YZF, s);
    r = launch_yz_fwd(Ly, y, s);
    if (r < 0) CKL(r);
  }
  if (r == 1) {  // the target plane: partial sums added, inverse y transform
    Timed t(ctx, KIND_YINV, s);
    CKL(launch_yz_finish(Ly, y, s));
  }
  *yinv_done = r == 1;
  return TM_OK;
}

// direct z sum from the source planes [zi0, zi0 + nzi) fused with the inverse y
// transform of every design plane
int zy_adjoint(tm_ctx* ctx, const ConvSpec& cs, int zi0, int nzi, cudaStream_t s, bool yfwd_inside) {
  const int Ly = ctx->L[1];
  const long long P = ctx->P;
  ZYArgs z{};
  z.src = ctx->B;
  z.src_cstride = (long long)ctx->nz * Ly * P;
  z.src_zstride = (long long)Ly * P;
  z.out = ctx->A;
  z.out_cstride = (long long)ctx->nz * ctx->ny * P;
  z.out_zstride = (long long)ctx->ny * P;
  z.P = ctx->P;
  z.n_out = ctx->ny;
  z.nin = cs.nin;
  z.nout = cs.nout;
  for (int i = 0; i < cs.nin; i++) z.in_slot[i] = cs.bin[i];
  for (int o = 0; o < cs.nout; o++) {
    z.out_slot[o] = cs.aout[o];
    for (int i = 0; i < cs.nin; i++) {
      coef6(z.coef[o][i], cs.v[o], cs.u[i]);
      z.need[o][i] = 0;
      for (int c = 0; c < 6; c++)
        if (z.coef[o][i][c] != 0.0f) z.need[o][i] |= 1 << c;
    }
  }
  z.Tz = ctx->Tz;
  z.Tdz = (long long)(Ly / 2 + 1) * P;
  z.Tc = (long long)ctx->nz * z.Tdz;
  z.zin0 = zi0;
  z.nzin = nzi;
  z.zout0 = 0;
  z.nzout = ctx->nzd;
  z.tw = ctx->tw + ctx->L[0];
  z.status = ctx->dstat;
  z.zero_word = ctx->gmax;  // cleared for the chain-rule pass that follows (saves a memset between kernels)
  z.pdl = ctx->pdl;
  const int c1 = cs.nin == 1 && cs.nout == 1 ? one_component(z.need[0][0]) : -1;
  if (c1 >= 0) {
    int r;
    bool rebuilt;
    if ((r = scaled_component(ctx, 1, c1, z.coef[0][0][c1], s, &z.Ts, &rebuilt))) return r;
    z.nzin_total = ctx->nz;
    // the adjoint reads its first tensor slice before it waits for the preceding kernel:
    // after a rebuild it must start only once the scaling kernel has finished
    if (rebuilt) z.pdl = 0;
  }
  if (yfwd_inside) {  // the source plane as x spectra: rows y < ny of plane zi0 of A slot ain[0]
    z.gsrc = ctx->A + cs.ain[0] * ((long long)ctx->nz * ctx->ny * P) + (long long)zi0 * ctx->ny * P;
    z.n_src = ctx->ny;
  }
  Timed t(ctx, KIND_ZYA, s);
  const int r = launch_zy_adj(Ly, z, s);
  if (r < 0) CKL(r);
  ctx->gmax_zeroed = r == 1;
  return TM_OK;
}

// forward x pass of the magnetization: rho^p (constant M0, contracted later) -> A slot 0,
// or rho^p M0_c (varying M0) -> A slots 0, 1, 2. Returns the number of slots written.
int xfwd_rho(tm_ctx* ctx, const float* rho, cudaStream_t s, int* nslots) {
  XFwdArgs x{};
  x.rows = ctx->nzd * ctx->ny;
  x.nx = ctx->nx;
  x.P = ctx->P;
  x.src = ctx->m0_var ? SRC_RHO_M0 : SRC_RHO_POW;
  x.rho = rho;
  x.p = (float)ctx->p;
  x.M0v = ctx->M0v;
  x.M0v_cstride = design_cells(ctx);
  for (int c = 0; c < 3; c++) {
    x.comp[c] = c;
    x.out_slot[c] = c;
  }
  x.out = ctx->A;
  x.out_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
  x.tw = ctx->tw;
  *nslots = ctx->m0_var ? 3 : 1;
  x.pdl = ctx->pdl;
  x.status = ctx->dstat;
  if (ctx->pend_rho && ctx->pend_rho == rho && xfwd_fuses_step(ctx->L[0], x.src, *nslots)) {
    x.upd_rho = ctx->pend_rho;
    x.upd_G = ctx->pend_G;
    x.upd_alpha = ctx->pend_alpha;
    x.upd_normalize = ctx->pend_normalize;
    x.upd_gmax = ctx->gmax;
    ctx->pend_rho = nullptr;  // consumed
  }
  Timed t(ctx, KIND_XFWD, s);
  CKL(launch_xfwd(ctx->L[0], x, *nslots, s));
  return TM_OK;
}

// inverse x pass on design rows with the chain rule into G (+ max |G|); ncomp slots:
// 1 = already contracted with the constant M0; 3 = components x, y, z (varying M0)
int xinv_chain(tm_ctx* ctx, const float* rho, float* G, int ncomp, const int* slots, cudaStream_t s) {
  if (!ctx->gmax_zeroed) CK(cudaMemsetAsync(ctx->gmax, 0, sizeof(unsigned int), s));
  ctx->gmax_zeroed = false;
  XInvArgs x{};
  x.pdl = ctx->pdl;
  x.rows = ctx->nzd * ctx->ny;
  x.nx = ctx->nx;
  x.P = ctx->P;
  x.sink = SINK_CHAIN;
  x.ncomp = ncomp;
  for (int j = 0; j < ncomp; j++) {
    x.comp[j] = j;
    x.in_slot[j] = slots[j];
  }
  x.in = ctx->A;
  x.in_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
  x.rho = rho;
  x.M0v = ncomp > 1 ? ctx->M0v : nullptr;
  x.M0v_cstride = design_cells(ctx);
  x.p = (float)ctx->p;
  x.G = G;
  x.gmax = ctx->gmax;
  x.tw = ctx->tw;
  x.status = ctx->dstat;
  Timed t(ctx, KIND_XINV, s);
  CKL(launch_xinv(ctx->L[0], x, s));
  ctx->gmax_of = G;
  return TM_OK;
}

// Forward convolution of the magnetization into the requested components F (A slots 0..nF-1).
int forward_field(tm_ctx* ctx, const float* rho, int nF, const int* F, const int* ext, cudaStream_t s) {
  int r, nsl;
  if ((r = xfwd_rho(ctx, rho, s, &nsl))) return r;
  ConvSpec cs{};
  if (!ctx->m0_var) {  // one input rho^p with u = M0; outputs v = e_c
    cs.nin = 1;
    cs.ain[0] = 0;
    cs.bin[0] = kSlotsB - 1;  // outputs use B slots 0..nF-1
    cs.u[0] = ctx->M0c;
  } else {
    cs.nin = 3;
    for (int i = 0; i < 3; i++) {
      cs.ain[i] = i;
      cs.bin[i] = i;
      cs.u[i] = kUnit[i];
    }
  }
  cs.nout = nF;
  for (int o = 0; o < nF; o++) {
    cs.bout[o] = o;
    cs.aout[o] = o;
    cs.v[o] = kUnit[F[o]];
  }
  cs.ext = ext;
  cs.out_ext = ext != nullptr;
  return conv_yz(ctx, cs, ctx->nzd, ctx->nz, s);
}

}  // namespace

extern "C" {

const char* tm_version(void) { return "topomag 0.1 (sm_103a)"; }

int tm_create(tm_ctx** out, int device) {
  if (!out) return TM_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return TM_ERR_ARG;
  tm_ctx* ctx = new tm_ctx();
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->Jdev, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->gmax, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->Jcount, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(ctx->Jcount, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->ext, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->Jhost, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->dstat, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(ctx->dstat, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->hstat, sizeof(unsigned));
  if (e != cudaSuccess) {
    tm_destroy(ctx);
    return TM_ERR_CUDA;
  }
  *out = ctx;
  return TM_OK;
}

void tm_destroy(tm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  free_grid(ctx);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  cudaFree(ctx->Jdev);
  cudaFree(ctx->dstat);
  if (ctx->hstat) cudaFreeHost(ctx->hstat);
  cudaFree(ctx->gmax);
  cudaFree(ctx->Jcount);
  cudaFree(ctx->ext);
  cudaFree(ctx->stats);
  cudaFree(ctx->nbad);
  if (ctx->Jhost) cudaFreeHost(ctx->Jhost);
  delete ctx;
}

const char* tm_last_error(const tm_ctx* ctx) { return ctx ? ctx->err : "null context"; }

int tm_set_grid(tm_ctx* ctx, const int n_out[3], int nzd, const double cellsize[3]) {
  return tm_set_grid_lengths(ctx, n_out, nzd, cellsize, nullptr);
}

int tm_set_grid_lengths(tm_ctx* ctx, const int n_out[3], int nzd, const double cellsize[3], const int L_in[3]) {
  INJECT(ctx, "tm_set_grid");
  if (!ctx || !n_out || !cellsize) return fail(ctx, TM_ERR_ARG, "null argument");
  for (int a = 0; a < 3; a++) {
    if (n_out[a] < 4 || n_out[a] > kMaxL / 2)
      return fail(ctx, TM_ERR_SIZE, "n_out[%d] = %d outside [4, %d]", a, n_out[a], kMaxL / 2);
    if (!(cellsize[a] > 0.0) || !isfinite(cellsize[a])) return fail(ctx, TM_ERR_ARG, "cellsize[%d] must be > 0", a);
  }
  if (nzd < 1 || nzd > n_out[2]) return fail(ctx, TM_ERR_ARG, "nzd = %d outside [1, nz = %d]", nzd, n_out[2]);
  for (int a = 0; a < 3; a++)
    if (L_in && L_in[a] != 0 && (!supported_L(L_in[a]) || L_in[a] < 2 * n_out[a]))
      return fail(ctx, TM_ERR_SIZE, "L[%d] = %d is not a supported length >= 2 n = %d", a, L_in[a], 2 * n_out[a]);
  CK(cudaSetDevice(ctx->device));
  free_grid(ctx);
  ctx->nx = n_out[0];
  ctx->ny = n_out[1];
  ctx->nz = n_out[2];
  ctx->nzd = nzd;
  for (int a = 0; a < 3; a++) {
    ctx->d[a] = cellsize[a];
    ctx->L[a] = (L_in && L_in[a] != 0) ? L_in[a] : pick_length(n_out[a]);
    if (ctx->L[a] == 0) return fail(ctx, TM_ERR_SIZE, "no supported FFT length for n = %d", n_out[a]);
  }
  const int Lx = ctx->L[0], Ly = ctx->L[1], Lz = ctx->L[2];
  ctx->P = ((Lx / 2 + 1) + TB - 1) / TB * TB;
  const long long P = ctx->P;
  if (zpass_smem(Lz) > 227 * 1024) return fail(ctx, TM_ERR_SIZE, "Lz = %d too large for the z pass", Lz);

  CK(cudaMalloc(&ctx->A, (long long)kSlotsA * ctx->nz * ctx->ny * P * sizeof(float2)));
  CK(cudaMalloc(&ctx->B, (long long)kSlotsB * ctx->nz * Ly * P * sizeof(float2)));
  CK(cudaMalloc(&ctx->T, 6LL * (Lz / 2 + 1) * (Ly / 2 + 1) * P * sizeof(float)));
  CK(cudaMalloc(&ctx->Tz, 6LL * ctx->nz * (Ly / 2 + 1) * P * sizeof(float)));
  // twiddles W_L^m = exp(-2 pi i m / L) from float64 host values
  std::vector<float2> tw;
  for (int a = 0; a < 3; a++)
    for (int m = 0; m < ctx->L[a]; m++) {
      const double t = 2.0 * M_PI * (double)m / (double)ctx->L[a];
      tw.push_back(make_float2((float)cos(t), (float)(-sin(t))));
    }
  CK(cudaMalloc(&ctx->tw, tw.size() * sizeof(float2)));
  CK(cudaMemcpy(ctx->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
  // z-pass column order: ky and Ly - ky adjacent (both read the same folded tensor column)
  std::vector<int2> zc;
  for (int ky = 0; ky <= Ly / 2; ky++) {
    zc.push_back(make_int2(host_pos_of_k(Ly, ky), ky));
    if (ky > 0 && ky < Ly / 2) zc.push_back(make_int2(host_pos_of_k(Ly, Ly - ky), Ly - ky));
  }
  CK(cudaMalloc(&ctx->zcol, zc.size() * sizeof(int2)));
  CK(cudaMemcpy(ctx->zcol, zc.data(), zc.size() * sizeof(int2), cudaMemcpyHostToDevice));
  const int rpb = xobj_rows_per_block() < xinv_rows_per_block() ? xobj_rows_per_block() : xinv_rows_per_block();
  ctx->nJpart = 3 * ((ctx->nz * ctx->ny + rpb - 1) / rpb);
  CK(cudaMalloc(&ctx->Jpart, ctx->nJpart * sizeof(double)));
  ctx->have_grid = true;
  ctx->err[0] = 0;
  return TM_OK;
}

int tm_default_fft_length(int n) { return n >= 1 && n <= kMaxL / 2 ? pick_length(n) : 0; }

int tm_get_fft_lengths(const tm_ctx* ctx, int L[3]) {
  if (!ctx || !L) return TM_ERR_ARG;
  if (!ctx->have_grid) return TM_ERR_STATE;
  for (int a = 0; a < 3; a++) L[a] = ctx->L[a];
  return TM_OK;
}

int tm_set_penalty(tm_ctx* ctx, double p) {
  INJECT(ctx, "tm_set_penalty");
  if (!ctx) return TM_ERR_ARG;
  if (!(p >= 1.0) || !isfinite(p)) return fail(ctx, TM_ERR_ARG, "penalty p = %g must be >= 1", p);
  ctx->p = p;
  return TM_OK;
}

int tm_set_M0(tm_ctx* ctx, const float* M0_dev, const double M0_const[3], void* stream) {
  INJECT(ctx, "tm_set_M0");
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  CK(cudaSetDevice(ctx->device));
  if (M0_dev) {
    if (!ctx->M0v) CK(cudaMalloc(&ctx->M0v, 3 * design_cells(ctx) * sizeof(float)));
    CK(cudaMemcpyAsync(ctx->M0v, M0_dev, 3 * design_cells(ctx) * sizeof(float), cudaMemcpyDeviceToDevice,
                       S(stream)));
    ctx->m0_var = true;
    for (int c = 0; c < 3; c++) ctx->M0c[c] = 0.0;
  } else {
    if (!M0_const) return fail(ctx, TM_ERR_ARG, "M0_dev and M0_const both null");
    for (int c = 0; c < 3; c++) {
      if (!isfinite(M0_const[c])) return fail(ctx, TM_ERR_ARG, "M0_const not finite");
      ctx->M0c[c] = M0_const[c];
    }
    ctx->m0_var = false;
  }
  ctx->have_M0 = true;
  return TM_OK;
}

int tm_set_tensor(tm_ctx* ctx, void* stream) {
  INJECT(ctx, "tm_set_tensor");
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  CK(cudaSetDevice(ctx->device));
  int r = tensor_setup(ctx->nx, ctx->ny, ctx->nz, ctx->d, ctx->L[0], ctx->L[1], ctx->L[2], ctx->P, ctx->T, ctx->Tz,
                       nullptr, S(stream), ctx->err, sizeof(ctx->err));
  if (r != 0) return TM_ERR_CUDA;
  ctx->have_tensor = true;
  ctx->tensor_gen++;
  return TM_OK;
}

int tm_stray_field(tm_ctx* ctx, const float* rho, float* H, void* stream) {
  INJECT(ctx, "tm_stray_field");
  int r = check_ready(ctx);
  if (r) return r;
  if (!rho || !H) return fail(ctx, TM_ERR_ARG, "null array");
  cudaStream_t s = S(stream);
  const int F[3] = {0, 1, 2};
  if ((r = forward_field(ctx, rho, 3, F, nullptr, s))) return r;
  XInvArgs x{};
  x.rows = ctx->nz * ctx->ny;
  x.nx = ctx->nx;
  x.P = ctx->P;
  x.sink = SINK_FIELD;
  x.ncomp = 3;
  for (int j = 0; j < 3; j++) {
    x.comp[j] = j;
    x.in_slot[j] = j;
  }
  x.in = ctx->A;
  x.in_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
  x.H = H;
  x.H_cstride = out_cells(ctx);
  x.tw = ctx->tw;
  {
    Timed t(ctx, KIND_XINV, s);
    CKL(launch_xinv(ctx->L[0], x, s));
  }
  return TM_OK;
}

int tm_stray_field_adjoint(tm_ctx* ctx, const float* rho, const float* gH, float* dJdrho, void* stream) {
  INJECT(ctx, "tm_stray_field_adjoint");
  int r = check_ready(ctx);
  if (r) return r;
  if (!rho || !gH || !dJdrho) return fail(ctx, TM_ERR_ARG, "null array");
  cudaStream_t s = S(stream);
  XFwdArgs x{};
  x.rows = ctx->nz * ctx->ny;
  x.nx = ctx->nx;
  x.P = ctx->P;
  x.src = SRC_VECTOR;
  x.vec = gH;
  x.vec_cstride = out_cells(ctx);
  for (int c = 0; c < 3; c++) {
    x.comp[c] = c;
    x.out_slot[c] = c;
  }
  x.out = ctx->A;
  x.out_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
  x.tw = ctx->tw;
  {
    Timed t(ctx, KIND_XFWD, s);
    CKL(launch_xfwd(ctx->L[0], x, 3, s));
  }
  ConvSpec cs{};
  cs.nin = 3;
  for (int i = 0; i < 3; i++) {
    cs.ain[i] = i;
    cs.bin[i] = i;
    cs.u[i] = kUnit[i];
  }
  const int slots[3] = {0, 1, 2};
  if (!ctx->m0_var) {  // contract the output with M0: one spectrum
    cs.nout = 1;
    cs.bout[0] = 0;
    cs.aout[0] = 0;
    cs.v[0] = ctx->M0c;
    if ((r = conv_yz(ctx, cs, ctx->nz, ctx->nzd, s))) return r;
    return xinv_chain(ctx, rho, dJdrho, 1, slots, s);
  }
  cs.nout = 3;
  for (int o = 0; o < 3; o++) {
    cs.bout[o] = o;
    cs.aout[o] = o;
    cs.v[o] = kUnit[o];
  }
  if ((r = conv_yz(ctx, cs, ctx->nz, ctx->nzd, s))) return r;
  return xinv_chain(ctx, rho, dJdrho, 3, slots, s);
}

int tm_objective_and_gradient(tm_ctx* ctx, const float* rho, const uint8_t* mask, const float* H_target,
                              const float Ht_const[3], const float w[3], double* J_host, float* dJdrho,
                              float* H_out, void* stream) {
  INJECT(ctx, "tm_objective_and_gradient");
  int r = check_ready(ctx);
  if (r) return r;
  if (!rho || !mask || !w || !dJdrho) return fail(ctx, TM_ERR_ARG, "null array");
  if (!H_target && !Ht_const) return fail(ctx, TM_ERR_ARG, "H_target and Ht_const both null");
  for (int c = 0; c < 3; c++)
    if (!isfinite(w[c])) return fail(ctx, TM_ERR_ARG, "weights must be finite");
  cudaStream_t s = S(stream);
  // components the objective weighs; the forward computes those (all three when H is
  // requested or M0 varies, because the varying-M0 chain rule needs every component)
  int W[3], nW = 0;
  for (int c = 0; c < 3; c++)
    if (w[c] != 0.0f) W[nW++] = c;
  const bool all3 = H_out || ctx->m0_var || nW == 0;
  int F[3], nF = 0;
  for (int c = 0; c < 3; c++)
    if (all3 || w[c] != 0.0f) F[nF++] = c;
  // without H_out only the planes holding target cells are needed: the forward
  // field is evaluated there alone and the adjoint source lives there alone
  const int* ext = nullptr;
  if (!H_out) {
    Timed t(ctx, KIND_OTHER, s);
    CKL(launch_mask_extent(mask, ctx->nz, (long long)ctx->ny * ctx->nx, ctx->ext, s));
    ext = ctx->ext;
  }
  if ((r = forward_field(ctx, rho, nF, F, ext, s))) return r;
  XInvArgs x{};
  x.rows = ctx->nz * ctx->ny;
  x.nx = ctx->nx;
  x.P = ctx->P;
  x.sink = SINK_OBJECTIVE;
  x.ncomp = nF;
  for (int j = 0; j < nF; j++) {
    x.comp[j] = F[j];
    x.in_slot[j] = j;
  }
  x.in = ctx->A;
  x.in_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
  x.H = H_out;
  x.H_cstride = out_cells(ctx);
  x.mask = mask;
  x.Ht = H_target;
  x.Ht_cstride = out_cells(ctx);
  for (int c = 0; c < 3; c++) {
    x.Htc[c] = Ht_const ? Ht_const[c] : 0.0f;
    x.w[c] = w[c];
  }
  x.adj_out = ctx->A;
  x.Jpart = ctx->Jpart;
  x.ext = ext;
  x.ny = ctx->ny;
  x.tw = ctx->tw;
  {
    Timed t(ctx, KIND_XINV, s);
    CKL(launch_xinv(ctx->L[0], x, s));
  }
  {
    Timed t(ctx, KIND_OTHER, s);
    const int nblk = (x.rows + xinv_rows_per_block() - 1) / xinv_rows_per_block();
    CKL(launch_j_finalize(ctx->Jpart, nF * nblk, ctx->Jdev, s));
  }
  // adjoint: sources g_c in the A slots of the forward outputs
  ConvSpec cs{};
  int slots[3] = {0, 1, 2};
  if (nW == 0) {
    CK(cudaMemsetAsync(dJdrho, 0, design_cells(ctx) * sizeof(float), s));
    ctx->gmax_of = nullptr;
  } else if (!ctx->m0_var) {  // inputs: weighted components; output contracted with M0
    cs.nin = nW;
    for (int i = 0; i < nW; i++) {
      int j = 0;
      while (F[j] != W[i]) j++;
      cs.ain[i] = j;
      cs.bin[i] = j;
      cs.u[i] = kUnit[W[i]];
    }
    cs.nout = 1;
    cs.bout[0] = cs.bin[0];
    cs.aout[0] = cs.ain[0];
    cs.v[0] = ctx->M0c;
    cs.ext = ext;
    cs.in_ext = ext != nullptr;
    if ((r = conv_yz(ctx, cs, ctx->nz, ctx->nzd, s))) return r;
    slots[0] = cs.aout[0];
    if ((r = xinv_chain(ctx, rho, dJdrho, 1, slots, s))) return r;
  } else {  // varying M0: all three components in and out
    cs.nin = 3;
    cs.nout = 3;
    for (int i = 0; i < 3; i++) {
      cs.ain[i] = cs.bin[i] = cs.bout[i] = cs.aout[i] = i;
      cs.u[i] = cs.v[i] = kUnit[i];
    }
    cs.ext = ext;
    cs.in_ext = ext != nullptr;
    if ((r = conv_yz(ctx, cs, ctx->nz, ctx->nzd, s))) return r;
    if ((r = xinv_chain(ctx, rho, dJdrho, 3, slots, s))) return r;
  }
  if (J_host) {
    CK(cudaMemcpyAsync(ctx->Jhost, ctx->Jdev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *J_host = *ctx->Jhost;
  }
  return TM_OK;
}

int tm_set_target(tm_ctx* ctx, const uint8_t* mask, const float* H_target, const float Ht_const[3], const float w[3],
                  void* stream) {
  INJECT(ctx, "tm_set_target");
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  if (!mask || !w) return fail(ctx, TM_ERR_ARG, "null array");
  if (!H_target && !Ht_const) return fail(ctx, TM_ERR_ARG, "H_target and Ht_const both null");
  for (int c = 0; c < 3; c++)
    if (!isfinite(w[c])) return fail(ctx, TM_ERR_ARG, "weights must be finite");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = S(stream);
  const long long n = out_cells(ctx);
  if (!ctx->tmask) CK(cudaMalloc(&ctx->tmask, n));
  CK(cudaMemcpyAsync(ctx->tmask, mask, n, cudaMemcpyDeviceToDevice, s));
  if (H_target) {
    if (!ctx->tHt) CK(cudaMalloc(&ctx->tHt, 3 * n * sizeof(float)));
    CK(cudaMemcpyAsync(ctx->tHt, H_target, 3 * n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  } else {
    cudaFree(ctx->tHt);
    ctx->tHt = nullptr;
  }
  for (int c = 0; c < 3; c++) {
    ctx->tHtc[c] = Ht_const ? Ht_const[c] : 0.0f;
    ctx->tw_[c] = w[c];
  }
  CKL(launch_mask_extent(ctx->tmask, ctx->nz, (long long)ctx->ny * ctx->nx, ctx->ext, s));
  int ext[2];
  CK(cudaMemcpyAsync(ext, ctx->ext, sizeof(ext), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ctx->tz0 = ext[1] > ext[0] ? ext[0] : 0;
  ctx->tz1 = ext[1] > ext[0] ? ext[1] : 0;
  ctx->have_target = true;
  ctx->target_kind = 0;
  return TM_OK;
}

namespace {

// Forward restricted to the target planes [tz0, tz1): x and y on the design planes,
// z summed directly onto the target planes, inverse y there. Field components F
// end up in A slots 0..nF-1 (half spectra along x).
int forward_planes(tm_ctx* ctx, const float* rho, const int* F, int nF, cudaStream_t s) {
  int r, nsl;
  const int np = ctx->tz1 - ctx->tz0;
  if ((r = xfwd_rho(ctx, rho, s, &nsl))) return r;
  ConvSpec cs{};
  cs.nin = nsl;
  for (int i = 0; i < nsl; i++) {
    cs.ain[i] = i;
    cs.bin[i] = i;
    cs.u[i] = nsl == 1 ? ctx->M0c : kUnit[i];
  }
  cs.nout = nF;
  for (int o = 0; o < nF; o++) {
    cs.bout[o] = o;
    cs.aout[o] = o;
    cs.v[o] = kUnit[F[o]];
  }
  if (ctx->fuse_yz && np == 1 && nF == 1) {
    bool done = false;
    if ((r = yz_forward(ctx, cs, ctx->tz0, s, &done))) return r;
    if (done) return TM_OK;
  } else {
    if ((r = ypass(ctx, false, cs.nin, cs.ain, cs.bin, 0, ctx->nzd, s))) return r;
    if ((r = zdirect(ctx, cs, 0, ctx->nzd, ctx->tz0, np, s))) return r;
  }
  return ypass(ctx, true, cs.nout, cs.aout, cs.bout, ctx->tz0, np, s);
}

// Adjoint from the target planes: slot j of A holds (x-transformed) dJ/dH of
// component F[j] on the target planes; the W components carry a source. y there,
// z summed directly onto the design planes, y and x inverse with the chain rule.
int adjoint_planes(tm_ctx* ctx, const float* rho, float* dJdrho, const int* F, const int* W, int nW,
                   cudaStream_t s) {
  int r;
  const int np = ctx->tz1 - ctx->tz0;
  ConvSpec ca{};
  if (!ctx->m0_var) {
    ca.nin = nW;
    for (int i = 0; i < nW; i++) {
      int j = 0;
      while (F[j] != W[i]) j++;
      ca.ain[i] = j;
      ca.bin[i] = j;
      ca.u[i] = kUnit[W[i]];
    }
    ca.nout = 1;
    ca.bout[0] = ca.bin[0];
    ca.aout[0] = ca.ain[0];
    ca.v[0] = ctx->M0c;
  } else {
    ca.nin = ca.nout = 3;
    for (int i = 0; i < 3; i++) {
      ca.ain[i] = ca.bin[i] = ca.bout[i] = ca.aout[i] = i;
      ca.u[i] = ca.v[i] = kUnit[i];
    }
  }
  // fused only in its single-spectrum, single-component form; with several spectra or
  // tensor components the separate passes measured faster
  bool simple = ca.nin == 1 && ca.nout == 1 && np == 1;
  if (simple) {
    float c6[6];
    coef6(c6, ca.v[0], ca.u[0]);
    int nc = 0;
    for (int c = 0; c < 6; c++) nc += c6[c] != 0.0f;
    simple = nc == 1;
  }
  // on the warp-specialized path the fused adjoint runs the source's y transform itself;
  // it then reads the source rows from A while it writes the design planes into A, so its
  // output goes to another slot (the target plane may be a design plane)
  const bool yfwd_inside = ctx->fuse_yz && simple && zy_adj_ws_length(ctx->L[1]) && ctx->ny <= ctx->L[1] / 2;
  if (yfwd_inside) ca.aout[0] = (ca.ain[0] + 1) % kSlotsA;
  if (!yfwd_inside && (r = ypass(ctx, false, ca.nin, ca.ain, ca.bin, ctx->tz0, np, s))) return r;
  if (ctx->fuse_yz && simple) {
    if ((r = zy_adjoint(ctx, ca, ctx->tz0, np, s, yfwd_inside))) return r;
  } else {
    if ((r = zdirect(ctx, ca, ctx->tz0, np, 0, ctx->nzd, s))) return r;
    if ((r = ypass(ctx, true, ca.nout, ca.aout, ca.bout, 0, ctx->nzd, s))) return r;
  }
  return xinv_chain(ctx, rho, dJdrho, ca.nout, ca.aout, s);
}

StencilArgs stencil_args(tm_ctx* ctx) {
  StencilArgs a{};
  a.K = ctx->sK;
  a.U = ctx->sU;
  a.rp = ctx->s_rp;
  a.idx = ctx->s_idx;
  a.a = ctx->s_a;
  a.c = ctx->s_c;
  a.cp = ctx->s_cp;
  a.cidx = ctx->s_cidx;
  a.crow = ctx->s_crow;
  a.ca = ctx->s_ca;
  a.H = ctx->sH;
  a.gH = ctx->sgH;
  a.r = ctx->s_r;
  a.part = ctx->s_part;
  a.J = ctx->Jdev;
  const long long b = (ctx->sK + 255) / 256;
  a.nblk = (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
  return a;
}

// J and dJ/drho of the prepared stencil objective
int evaluate_stencil(tm_ctx* ctx, const float* rho, float* dJdrho, cudaStream_t s) {
  int r;
  int W[3], nW = 0;
  for (int c = 0; c < 3; c++)
    if (ctx->s_comps & (1 << c)) W[nW++] = c;
  const int np = ctx->tz1 - ctx->tz0;
  if (ctx->sK == 0 || nW == 0) {
    CK(cudaMemsetAsync(ctx->Jdev, 0, sizeof(double), s));
    CK(cudaMemsetAsync(dJdrho, 0, design_cells(ctx) * sizeof(float), s));
    ctx->gmax_of = nullptr;
    return TM_OK;
  }
  const StencilArgs sa = stencil_args(ctx);
  if (np > kDirectPlanesMax) {  // many planes: full field, then the full adjoint
    if ((r = tm_stray_field(ctx, rho, ctx->sH, s))) return r;
    {
      Timed t(ctx, KIND_OTHER, s);
      CKL(launch_stencil(sa, s));
    }
    return tm_stray_field_adjoint(ctx, rho, ctx->sgH, dJdrho, s);
  }
  int F[3], nF = 0;
  for (int c = 0; c < 3; c++)
    if (ctx->m0_var || (ctx->s_comps & (1 << c))) F[nF++] = c;
  if ((r = forward_planes(ctx, rho, F, nF, s))) return r;
  {  // H of the F components on the target planes
    XInvArgs x{};
    x.row_base = ctx->tz0 * ctx->ny;
    x.rows = ctx->tz1 * ctx->ny;
    x.nx = ctx->nx;
    x.P = ctx->P;
    x.sink = SINK_FIELD;
    x.ncomp = nF;
    for (int j = 0; j < nF; j++) {
      x.comp[j] = F[j];
      x.in_slot[j] = j;
    }
    x.in = ctx->A;
    x.in_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
    x.H = ctx->sH;
    x.H_cstride = out_cells(ctx);
    x.tw = ctx->tw;
    Timed t(ctx, KIND_XINV, s);
    CKL(launch_xinv(ctx->L[0], x, s));
  }
  {
    Timed t(ctx, KIND_OTHER, s);
    CKL(launch_stencil(sa, s));
  }
  {  // dJ/dH on the target planes, transformed along x into the same slots
    const long long plane = (long long)ctx->ny * ctx->nx;
    XFwdArgs x{};
    x.rows = np * ctx->ny;
    x.nx = ctx->nx;
    x.P = ctx->P;
    x.src = SRC_VECTOR;
    x.vec = ctx->sgH + ctx->tz0 * plane;
    x.vec_cstride = out_cells(ctx);
    for (int j = 0; j < nF; j++) {
      x.comp[j] = F[j];
      x.out_slot[j] = j;
    }
    x.out = ctx->A + (long long)ctx->tz0 * ctx->ny * ctx->P;
    x.out_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
    x.tw = ctx->tw;
    Timed t(ctx, KIND_XFWD, s);
    CKL(launch_xfwd(ctx->L[0], x, nF, s));
  }
  return adjoint_planes(ctx, rho, dJdrho, F, W, nW, s);
}

}  // namespace

int tm_set_stencil_objective(tm_ctx* ctx, long long K, const long long* row_ptr, const int* comp,
                             const long long* cell, const double* a, const double* c, void* stream) {
  INJECT(ctx, "tm_set_stencil_objective");
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  if (K < 0 || (K > 0 && (!row_ptr || !comp || !cell || !a || !c))) return fail(ctx, TM_ERR_ARG, "null array");
  if (K > 0x7fffffffLL) return fail(ctx, TM_ERR_SIZE, "too many rows");
  const long long ocells = out_cells(ctx), plane = (long long)ctx->ny * ctx->nx;
  const long long E = K > 0 ? row_ptr[K] : 0;
  if (K > 0 && row_ptr[0] != 0) return fail(ctx, TM_ERR_ARG, "row_ptr[0] must be 0");
  for (long long k = 0; k < K; k++) {
    if (row_ptr[k + 1] < row_ptr[k]) return fail(ctx, TM_ERR_ARG, "row_ptr must not decrease");
    if (!isfinite(c[k])) return fail(ctx, TM_ERR_ARG, "row weights must be finite");
  }
  int comps = 0, z0 = ctx->nz, z1 = 0;
  std::vector<long long> idx(E);
  for (long long e = 0; e < E; e++) {
    if (comp[e] < 0 || comp[e] > 2 || cell[e] < 0 || cell[e] >= ocells || !isfinite(a[e]))
      return fail(ctx, TM_ERR_ARG, "entry %lld: component, cell or coefficient out of range", e);
    idx[e] = comp[e] * ocells + cell[e];
    comps |= 1 << comp[e];
    const int z = (int)(cell[e] / plane);
    z0 = z < z0 ? z : z0;
    z1 = z + 1 > z1 ? z + 1 : z1;
  }
  // column form: entries ordered by value index, then by row
  std::vector<long long> rowof(E), ord(E);
  for (long long k = 0; k < K; k++)
    for (long long e = row_ptr[k]; e < row_ptr[k + 1]; e++) rowof[e] = k;
  for (long long e = 0; e < E; e++) ord[e] = e;
  std::stable_sort(ord.begin(), ord.end(), [&](long long x, long long y) { return idx[x] < idx[y]; });
  std::vector<long long> cp, cidx;
  std::vector<int> crow(E);
  std::vector<double> ca(E);
  for (long long q = 0; q < E; q++) {
    const long long e = ord[q];
    if (q == 0 || idx[e] != idx[ord[q - 1]]) {
      cp.push_back(q);
      cidx.push_back(idx[e]);
    }
    crow[q] = (int)rowof[e];
    ca[q] = a[e];
  }
  cp.push_back(E);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = S(stream);
  free_stencil(ctx);
  const size_t fb = 3 * (size_t)ocells * sizeof(float);
  if (!ctx->sH) CK(cudaMalloc(&ctx->sH, fb));
  if (!ctx->sgH) CK(cudaMalloc(&ctx->sgH, fb));
  CK(cudaMemsetAsync(ctx->sgH, 0, fb, s));
  const long long U = (long long)cidx.size();
  auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, bytes > 0 ? bytes : 8);
    if (e == cudaSuccess && bytes > 0) e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s);
    return e;
  };
  CK(up((void**)&ctx->s_rp, row_ptr, K > 0 ? (K + 1) * sizeof(long long) : 0));
  CK(up((void**)&ctx->s_idx, idx.data(), E * sizeof(long long)));
  CK(up((void**)&ctx->s_a, a, E * sizeof(double)));
  CK(up((void**)&ctx->s_c, c, K * sizeof(double)));
  CK(up((void**)&ctx->s_cp, cp.data(), cp.size() * sizeof(long long)));
  CK(up((void**)&ctx->s_cidx, cidx.data(), U * sizeof(long long)));
  CK(up((void**)&ctx->s_crow, crow.data(), E * sizeof(int)));
  CK(up((void**)&ctx->s_ca, ca.data(), E * sizeof(double)));
  CK(cudaMalloc(&ctx->s_r, (K > 0 ? K : 1) * sizeof(double)));
  CK(cudaMalloc(&ctx->s_part, 1024 * sizeof(double)));
  CK(cudaStreamSynchronize(s));  // the host arrays above are released on return
  ctx->sK = K;
  ctx->sU = U;
  ctx->s_comps = comps;
  ctx->tz0 = E > 0 ? z0 : 0;
  ctx->tz1 = E > 0 ? z1 : 0;
  ctx->target_kind = 1;
  ctx->have_target = true;
  return TM_OK;
}

int tm_evaluate(tm_ctx* ctx, const float* rho, double* J_host, float* dJdrho, void* stream) {
  INJECT(ctx, "tm_evaluate");
  int r = check_ready(ctx);
  if (r) return r;
  if (!ctx->have_target) return fail(ctx, TM_ERR_STATE, "no target: call tm_set_target first");
  if (!rho || !dJdrho) return fail(ctx, TM_ERR_ARG, "null array");
  cudaStream_t s = S(stream);
  if (ctx->target_kind == 1) {
    if ((r = evaluate_stencil(ctx, rho, dJdrho, s))) return r;
  } else {
    const int np = ctx->tz1 - ctx->tz0;
    if (np > kDirectPlanesMax)  // many target planes: the FFT z pass is cheaper
      return tm_objective_and_gradient(ctx, rho, ctx->tmask, ctx->tHt, ctx->tHtc, ctx->tw_, J_host, dJdrho,
                                       nullptr, stream);
    const float* w = ctx->tw_;
    int W[3], nW = 0;
    for (int c = 0; c < 3; c++)
      if (w[c] != 0.0f) W[nW++] = c;
    if (np == 0 || nW == 0) {
      CK(cudaMemsetAsync(ctx->Jdev, 0, sizeof(double), s));
      CK(cudaMemsetAsync(dJdrho, 0, design_cells(ctx) * sizeof(float), s));
    ctx->gmax_of = nullptr;
    } else {
      int F[3], nF = 0;
      for (int c = 0; c < 3; c++)
        if (ctx->m0_var || w[c] != 0.0f) F[nF++] = c;
      if ((r = forward_planes(ctx, rho, F, nF, s))) return r;
      // objective on the target rows; dJ/dH transformed along x in place
      XInvArgs x{};
      x.row_base = ctx->tz0 * ctx->ny;
      x.rows = ctx->tz1 * ctx->ny;
      x.nx = ctx->nx;
      x.P = ctx->P;
      x.sink = SINK_OBJECTIVE;
      x.ncomp = nF;
      for (int j = 0; j < nF; j++) {
        x.comp[j] = F[j];
        x.in_slot[j] = j;
      }
      x.in = ctx->A;
      x.in_cstride = (long long)ctx->nz * ctx->ny * ctx->P;
      x.H_cstride = out_cells(ctx);
      x.mask = ctx->tmask;
      x.Ht = ctx->tHt;
      x.Ht_cstride = out_cells(ctx);
      for (int c = 0; c < 3; c++) {
        x.Htc[c] = ctx->tHtc[c];
        x.w[c] = w[c];
      }
      x.adj_out = ctx->A;
      x.Jpart = ctx->Jpart;
      x.Jcount = ctx->Jcount;  // J summed by the pass's last block
      x.Jout = ctx->Jdev;
      x.ny = ctx->ny;
      x.tw = ctx->tw;
      x.pdl = ctx->pdl;
      {  // few target rows: the latency-bound compact kernel (one warp group per row pair)
        Timed t(ctx, KIND_OBJ, s);
        CKL(launch_xobj(ctx->L[0], x, s));
      }
      if ((r = adjoint_planes(ctx, rho, dJdrho, F, W, nW, s))) return r;
    }
  }
  if (J_host) {
    CK(cudaMemcpyAsync(ctx->Jhost, ctx->Jdev, sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((r = check_status(ctx, s))) return r;  // synchronises s
    *J_host = *ctx->Jhost;
  }
  return TM_OK;
}

int tm_get_objective(tm_ctx* ctx, double* J_host, void* stream) {
  INJECT(ctx, "tm_get_objective");
  if (!ctx || !J_host) return fail(ctx, TM_ERR_ARG, "null argument");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpyAsync(ctx->Jhost, ctx->Jdev, sizeof(double), cudaMemcpyDeviceToHost, S(stream)));
  int r = check_status(ctx, S(stream));  // synchronises the stream
  if (r) return r;
  *J_host = *ctx->Jhost;
  return TM_OK;
}

int tm_copy_objective(tm_ctx* ctx, double* dst, void* stream) {
  INJECT(ctx, "tm_copy_objective");
  if (!ctx || !dst) return fail(ctx, TM_ERR_ARG, "null argument");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpyAsync(dst, ctx->Jdev, sizeof(double), cudaMemcpyDefault, S(stream)));
  return TM_OK;
}

int tm_optimize_step(tm_ctx* ctx, float* rho, const float* dJdrho, float alpha, int normalize, void* stream) {
  INJECT(ctx, "tm_optimize_step");
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  if (!rho || !dJdrho) return fail(ctx, TM_ERR_ARG, "null array");
  if (!isfinite(alpha)) return fail(ctx, TM_ERR_ARG, "alpha not finite");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = S(stream);
  const long long n = design_cells(ctx);
  Timed t(ctx, KIND_OTHER, s);
  // normalize 2: reuse max|G| of the evaluation that wrote dJdrho (the caller has not changed it)
  if (normalize && !(normalize == 2 && ctx->gmax_of == dJdrho)) {
    CK(cudaMemsetAsync(ctx->gmax, 0, sizeof(unsigned int), s));
    CKL(launch_absmax(dJdrho, n, ctx->gmax, s));
    ctx->gmax_of = dJdrho;
  }
  CKL(launch_update(rho, dJdrho, n, alpha, normalize != 0, ctx->gmax, s));
  return TM_OK;
}

int tm_evaluate_step(tm_ctx* ctx, float* rho, float alpha, int normalize, double* J_host, float* dJdrho,
                     void* stream) {
  INJECT(ctx, "tm_evaluate_step");
  int r = check_ready(ctx);
  if (r) return r;
  if (!ctx->have_target) return fail(ctx, TM_ERR_STATE, "no target: call tm_set_target first");
  if (!rho || !dJdrho) return fail(ctx, TM_ERR_ARG, "null array");
  if (!isfinite(alpha)) return fail(ctx, TM_ERR_ARG, "alpha not finite");
  cudaStream_t s = S(stream);
  const long long n = design_cells(ctx);
  if (normalize && !(normalize == 2 && ctx->gmax_of == dJdrho)) {
    Timed t(ctx, KIND_OTHER, s);
    CK(cudaMemsetAsync(ctx->gmax, 0, sizeof(unsigned int), s));
    CKL(launch_absmax(dJdrho, n, ctx->gmax, s));
    ctx->gmax_of = dJdrho;
  }
  // the step runs inside the x forward pass of rho when the prepared path reaches it with
  // one spectrum; otherwise as its own pass first
  const int np = ctx->tz1 - ctx->tz0;
  int nW = 0;
  for (int c = 0; c < 3; c++) nW += ctx->tw_[c] != 0.0f;
  const bool fused = ctx->target_kind == 0 && np >= 1 && np <= kDirectPlanesMax && nW > 0 &&
                     (reinterpret_cast<uintptr_t>(dJdrho) & 15) == 0 &&  // copied in 16-byte pieces
                     xfwd_fuses_step(ctx->L[0], ctx->m0_var ? SRC_RHO_M0 : SRC_RHO_POW, ctx->m0_var ? 3 : 1);
  if (fused) {
    ctx->pend_rho = rho;
    ctx->pend_G = dJdrho;
    ctx->pend_alpha = alpha;
    ctx->pend_normalize = normalize != 0;
  } else {
    Timed t(ctx, KIND_OTHER, s);
    CKL(launch_update(rho, dJdrho, n, alpha, normalize != 0, ctx->gmax, s));
  }
  r = tm_evaluate(ctx, rho, J_host, dJdrho, stream);
  if (ctx->pend_rho) {
    ctx->pend_rho = nullptr;
    if (!r) return fail(ctx, TM_ERR_STATE, "internal: the pending step was not applied");
  }
  return r;
}

int tm_check_design(tm_ctx* ctx, const float* rho, long long* n_bad, void* stream) {
  INJECT(ctx, "tm_check_design");
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  if (!rho || !n_bad) return fail(ctx, TM_ERR_ARG, "null argument");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = S(stream);
  if (!ctx->nbad) CK(cudaMalloc(&ctx->nbad, sizeof(unsigned long long)));
  CK(cudaMemsetAsync(ctx->nbad, 0, sizeof(unsigned long long), s));
  CKL(launch_check_design(rho, design_cells(ctx), ctx->nbad, s));
  unsigned long long nb = 0;
  CK(cudaMemcpyAsync(&nb, ctx->nbad, sizeof(nb), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *n_bad = (long long)nb;
  if (nb) return fail(ctx, TM_ERR_ARG, "rho: %llu of %lld entries are NaN or outside [0, 1]", nb, design_cells(ctx));
  return TM_OK;
}

int tm_iteration_stats(tm_ctx* ctx, const float* rho, const float* dJdrho, double out[3], void* stream) {
  INJECT(ctx, "tm_iteration_stats");
  if (!ctx) return TM_ERR_ARG;
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  if (!rho || !dJdrho || !out) return fail(ctx, TM_ERR_ARG, "null argument");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = S(stream);
  constexpr int kStatBlocks = 512;
  if (!ctx->stats) CK(cudaMalloc(&ctx->stats, (2 * kStatBlocks + 2) * sizeof(double)));
  const long long n = design_cells(ctx);
  if (ctx->gmax_of != dJdrho) {  // max|G| of this array (the evaluation that wrote it keeps it otherwise)
    CK(cudaMemsetAsync(ctx->gmax, 0, sizeof(unsigned int), s));
    CKL(launch_absmax(dJdrho, n, ctx->gmax, s));
    ctx->gmax_of = dJdrho;
  }
  CKL(launch_rho_stats(rho, n, ctx->stats, kStatBlocks, ctx->stats + 2 * kStatBlocks, s));
  double h[2];
  unsigned gbits = 0;
  CK(cudaMemcpyAsync(h, ctx->stats + 2 * kStatBlocks, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&gbits, ctx->gmax, sizeof(gbits), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float gm;
  memcpy(&gm, &gbits, sizeof(gm));
  out[0] = gm;
  out[1] = h[0] / (double)n;
  out[2] = h[1] / (double)n;
  return TM_OK;
}

int tm_inject_fault(const char* call, long long nth) {
  Injection& in = injection();
  std::lock_guard<std::mutex> lock(in.mu);
  if (!call || nth <= 0) {
    in.call.clear();
    in.left = 0;
    return TM_OK;
  }
  in.call = call;
  in.left = nth;
  return TM_OK;
}

int tm_selftest_wait_timeout(tm_ctx* ctx, int polls, void* stream) {
  INJECT(ctx, "tm_selftest_wait_timeout");
  if (!ctx) return TM_ERR_ARG;
  if (polls < 1 || polls > 65536) return fail(ctx, TM_ERR_ARG, "polls = %d outside [1, 65536]", polls);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = S(stream);
  CKL(launch_wait_selftest(ctx->dstat, polls, s));
  const int r = check_status(ctx, s);
  if (r == TM_OK) return fail(ctx, TM_ERR_CUDA, "the self-test wait did not set the status word");
  return r;
}

int tm_set_fused(tm_ctx* ctx, int on) {
  INJECT(ctx, "tm_set_fused");
  if (!ctx) return TM_ERR_ARG;
  ctx->fuse_yz = on != 0;
  return TM_OK;
}

int tm_profile(tm_ctx* ctx, int on) {
  INJECT(ctx, "tm_profile");
  if (!ctx) return TM_ERR_ARG;
  ctx->prof_on = on != 0;
  ctx->ev_used = 0;
  return TM_OK;
}

int tm_profile_read(tm_ctx* ctx, double ms[9], int launches[9]) {
  INJECT(ctx, "tm_profile_read");
  if (!ctx || !ms || !launches) return fail(ctx, TM_ERR_ARG, "null argument");
  CK(cudaSetDevice(ctx->device));
  for (int k = 0; k < KIND_N; k++) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (size_t i = 0; i < ctx->ev_used; i++) {
    CK(cudaEventSynchronize(ctx->ev[2 * i + 1]));
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    ms[ctx->ev_kind[i]] += t;
    launches[ctx->ev_kind[i]] += 1;
  }
  return TM_OK;
}

int tm_debug_tensor_octant(tm_ctx* ctx, double* host_out, void* stream) {
  if (!ctx || !host_out) return fail(ctx, TM_ERR_ARG, "null argument");
  if (!ctx->have_grid) return fail(ctx, TM_ERR_STATE, "no grid: call tm_set_grid first");
  CK(cudaSetDevice(ctx->device));
  float* tmp = nullptr;
  CK(cudaMalloc(&tmp, 6LL * (ctx->L[2] / 2 + 1) * (ctx->L[1] / 2 + 1) * ctx->P * sizeof(float)));
  int r = tensor_setup(ctx->nx, ctx->ny, ctx->nz, ctx->d, ctx->L[0], ctx->L[1], ctx->L[2], ctx->P, tmp, nullptr,
                       host_out, S(stream), ctx->err, sizeof(ctx->err));
  cudaFree(tmp);
  return r ? TM_ERR_CUDA : TM_OK;
}

int tm_debug_tensor_spectrum(tm_ctx* ctx, float* host_out, void* stream) {
  if (!ctx || !host_out) return fail(ctx, TM_ERR_ARG, "null argument");
  if (!ctx->have_tensor) return fail(ctx, TM_ERR_STATE, "no tensor: call tm_set_tensor first");
  CK(cudaSetDevice(ctx->device));
  const int KX = ctx->L[0] / 2 + 1;
  const long long rows = 6LL * (ctx->L[2] / 2 + 1) * (ctx->L[1] / 2 + 1);
  CK(cudaMemcpy2DAsync(host_out, KX * sizeof(float), ctx->T, ctx->P * sizeof(float), KX * sizeof(float), rows,
                       cudaMemcpyDeviceToHost, S(stream)));
  CK(cudaStreamSynchronize(S(stream)));
  return TM_OK;
}

}  // extern "C"

namespace tmk {

int host_pos_of_k(int L, int k) {
  int pos = 0, span = L, rem = k;
  for (int s = 0; s < plan_stages(L); s++) {
    const int R = plan_radix(L, s);
    span /= R;
    pos += (rem % R) * span;
    rem /= R;
  }
  return pos;
}

int host_k_of_pos(int L, int pos) {
  const int S = plan_stages(L);
  int d[8];
  int rem = pos;
  for (int s = S - 1; s >= 0; s--) {
    d[s] = rem % plan_radix(L, s);
    rem /= plan_radix(L, s);
  }
  int k = 0, m = 1;
  for (int s = 0; s < S; s++) {
    k += d[s] * m;
    m *= plan_radix(L, s);
  }
  return k;
}

}  // namespace tmk
