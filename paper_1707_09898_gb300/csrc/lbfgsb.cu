// L-BFGS-B on the GPU (Byrd, Lu, Nocedal and Zhu 1995; projected subspace step of
// Morales and Nocedal 2011; More-Thuente line search), the bound-constrained
// quasi-Newton method the paper minimises its objective with (Sec.
// "Discretization"; Table I counts its iterations).
//
// Device (float64): iterate x, gradient g, direction d, Cauchy point xcp, subspace
// point xbar, the m correction pairs S, Y (one array of n per pair, a ring of
// slots), and every length-n operation. Host: the 2m x 2m middle matrix of the
// compact representation B = theta I - W M W^T, W = [Y, theta S] (oldest pair
// first), and the scalar line-search logic. Reductions write one partial per
// block and are summed in block order, so every run is bit-reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/topomag.h"
#include "../../include/topomag_lbfgsb.h"

namespace {

constexpr int MAXM = 16;  // 2m <= 32: one lane per column of W in the breakpoint scan
constexpr int NT = 256;
constexpr int WPB = NT / 32;
constexpr int TILE = 2048;  // elements per block in compaction and radix sort (8 per thread)
constexpr double EPSMCH = 2.220446049250313e-16;
constexpr double BIG = 1e10;

struct Cols {        // logical column k of [Y | S] (oldest first) -> storage slot
  int col;           // pairs in memory
  int slot[MAXM];
};

// W(a, i): a < col -> Y_a[i]; col <= a < 2 col -> theta * S_{a-col}[i]
__device__ __forceinline__ double wcol(const double* __restrict__ S, const double* __restrict__ Y, long long n,
                                       const Cols& c, double theta, int a, long long i) {
  return a < c.col ? Y[(long long)c.slot[a] * n + i] : theta * S[(long long)c.slot[a - c.col] * n + i];
}

// ---- block reductions: one partial per block, summed in block order later ----
template <int K>
__device__ void block_sums(double (&v)[K], int nv, double* part) {
  __shared__ double sh[WPB][K];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; k++) {
    if (k < nv) {
      double a = v[k];
      for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
      if (lane == 0) sh[w][k] = a;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nv; k += NT) {
    double s = 0.0;
    for (int i = 0; i < WPB; i++) s += sh[i][k];
    part[(long long)blockIdx.x * nv + k] = s;
  }
}

__global__ void k_finish(const double* part, int nblk, int nv, double* out) {
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += part[(long long)b * nv + k];
    out[k] = s;
  }
}

// min of (value, index) pairs: smaller value, then smaller index
struct VI {
  double v;
  long long i;
};
__device__ __forceinline__ VI vimin(VI a, VI b) { return (b.v < a.v || (b.v == a.v && b.i < a.i)) ? b : a; }
__device__ void block_min(VI x, VI* part) {
  __shared__ VI sh[WPB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) {
    VI y;
    y.v = __shfl_down_sync(0xffffffffu, x.v, o);
    y.i = __shfl_down_sync(0xffffffffu, x.i, o);
    x = vimin(x, y);
  }
  if (lane == 0) sh[w] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    VI r = sh[0];
    for (int i = 1; i < WPB; i++) r = vimin(r, sh[i]);
    part[blockIdx.x] = r;
  }
}
__global__ void k_finish_min(const VI* part, int nblk, VI* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    VI r = part[0];
    for (int b = 1; b < nblk; b++) r = vimin(r, part[b]);
    *out = r;
  }
}

// ---- start: x = P(x0) --------------------------------------------------------
__global__ void k_start(const float* x32, const double* x64, long long n, double lo, double hi, double* x,
                        float* e32, double* e64) {
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    double v = x64 ? x64[i] : (double)x32[i];
    v = fmin(fmax(v, lo), hi);
    x[i] = v;
    if (e32) e32[i] = (float)v;
    if (e64) e64[i] = v;
  }
}

// g = (double) gradient; sums: [0] gnew . d
__global__ void k_load_g(const float* g32, const double* g64, long long n, const double* d, double* g, double* part) {
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    const double gi = g64 ? g64[i] : (double)g32[i];
    g[i] = gi;
    if (d) v[0] += gi * d[i];
  }
  block_sums<1>(v, 1, part);
}

// projected gradient infinity norm of (x, g) as a max over blocks (as a "min" of -|.|)
__global__ void k_projgr(const double* x, const double* g, long long n, double lo, double hi, VI* part) {
  VI m{0.0, 0};
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    double gi = g[i];
    gi = gi < 0.0 ? fmax(x[i] - hi, gi) : fmin(x[i] - lo, gi);
    m = vimin(m, VI{-fabs(gi), i});
  }
  block_min(m, part);
}

// ---- generalized Cauchy point --------------------------------------------------
// Per variable: status (0 moving, 1 fixed at lower, 2 fixed at upper, 3 zero gradient),
// d = -g on moving variables, breakpoint t; block sums: p0 = W^T d (2 col), d.d; block
// counts of breakpoints (for the stable compaction).
__global__ void k_bp(const double* __restrict__ x, const double* __restrict__ g, long long n, double lo, double hi,
                     const double* __restrict__ S, const double* __restrict__ Y, Cols c, double theta,
                     double* __restrict__ d, double* __restrict__ t, int8_t* __restrict__ st, double* part,
                     int* cnt, VI* tmin) {
  VI tm{INFINITY, -1};
  double v[2 * MAXM + 1];
#pragma unroll
  for (int k = 0; k < 2 * MAXM + 1; k++) v[k] = 0.0;
  const int col2 = 2 * c.col;
  int count = 0;
  const long long base = (long long)blockIdx.x * TILE;
  for (int r = 0; r < TILE / NT; r++) {
    const long long i = base + r * NT + threadIdx.x;
    if (i >= n) break;
    const double xi = x[i], ng = -g[i];
    const double tl = xi - lo, tu = hi - xi;
    int s = 0;
    if (tl <= 0.0) {
      if (ng <= 0.0) s = 1;
    } else if (tu <= 0.0) {
      if (ng >= 0.0) s = 2;
    } else if (fabs(ng) <= 0.0) {
      s = 3;
    }
    double di = 0.0, ti = INFINITY;
    if (s == 0) {
      di = ng;
      ti = ng < 0.0 ? tl / (-ng) : tu / ng;
      tm = vimin(tm, VI{ti, i});
      count++;
#pragma unroll
      for (int a = 0; a < 2 * MAXM; a++)
        if (a < col2) v[a] += wcol(S, Y, n, c, theta, a, i) * di;
      v[2 * MAXM] += di * di;
    }
    d[i] = di;
    t[i] = ti;
    st[i] = (int8_t)s;
  }
  // d.d goes to slot col2 of the partial
  v[col2] = v[2 * MAXM];
  block_sums<2 * MAXM + 1>(v, col2 + 1, part);
  block_min(tm, tmin);
  for (int o = 16; o; o >>= 1) count += __shfl_down_sync(0xffffffffu, count, o);
  __shared__ int shc[WPB];
  if ((threadIdx.x & 31) == 0) shc[threadIdx.x >> 5] = count;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < WPB; w++) s += shc[w];
    cnt[blockIdx.x] = s;
  }
}

// exclusive scan of a (small) int array in one block; total in out[len]
__global__ void k_scan_ex(int* a, long long len) {
  __shared__ long long sh[1024];
  const int T = blockDim.x;
  const long long chunk = (len + T - 1) / T;
  const long long b0 = threadIdx.x * chunk, b1 = min(len, b0 + chunk);
  long long s = 0;
  for (long long i = b0; i < b1; i++) s += a[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int k = 0; k < T; k++) {
      const long long v = sh[k];
      sh[k] = run;
      run += v;
    }
    a[len] = (int)run;
  }
  __syncthreads();
  long long run = sh[threadIdx.x];
  for (long long i = b0; i < b1; i++) {
    const int v = a[i];
    a[i] = (int)run;
    run += v;
  }
}

// block-stable position of flagged elements, 256 per round
__device__ __forceinline__ int block_rank(bool f, int* shw, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned b = __ballot_sync(0xffffffffu, f);
  if (lane == 0) shw[w] = __popc(b);
  __syncthreads();
  int off = 0;
  total = 0;
  for (int k = 0; k < WPB; k++) {
    if (k < w) off += shw[k];
    total += shw[k];
  }
  __syncthreads();
  return off + __popc(b & ((1u << lane) - 1u));
}

// breakpoints compacted in index order: key = bits of t (t > 0, so bit order = value order)
__global__ void k_bp_compact(const double* t, const int8_t* st, long long n, const int* off, unsigned long long* key,
                             int* val) {
  __shared__ int shw[WPB];
  const long long base = (long long)blockIdx.x * TILE;
  int run = off[blockIdx.x];
  for (int r = 0; r < TILE / NT; r++) {
    const long long i = base + r * NT + threadIdx.x;
    const bool f = i < n && st[i] == 0;
    int total;
    const int pos = block_rank(f, shw, total);
    if (f) {
      key[run + pos] = (unsigned long long)__double_as_longlong(t[i]);
      val[run + pos] = (int)i;
    }
    run += total;
  }
}

// ---- LSD radix sort of (uint64 key, int value), 8 bits per pass, stable ----------
__global__ void k_rs_hist(const unsigned long long* key, int K, int shift, int* hist, int ntile) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * TILE;
  for (int r = 0; r < TILE / NT; r++) {
    const long long e = base + r * NT + threadIdx.x;
    if (e < K) atomicAdd(&h[(key[e] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[threadIdx.x * ntile + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const unsigned long long* key, const int* val, int K, int shift, const int* off,
                             int ntile, unsigned long long* key2, int* val2) {
  __shared__ int wc[WPB][256];
  __shared__ int run[256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = off[threadIdx.x * ntile + blockIdx.x];
  const long long base = (long long)blockIdx.x * TILE;
  for (int r = 0; r < TILE / NT; r++) {
    for (int k = 0; k < WPB; k++) wc[k][threadIdx.x] = 0;
    __syncthreads();
    const long long e = base + r * NT + threadIdx.x;
    const bool ok = e < K;
    const unsigned long long kk = ok ? key[e] : 0ull;
    const int dg = ok ? (int)((kk >> shift) & 255) : 256 + lane;  // invalid: unique per lane, never matched
    const unsigned mm = __match_any_sync(0xffffffffu, dg);
    const int rank = __popc(mm & ((1u << lane) - 1u));
    if (ok && rank == 0) wc[w][dg] = __popc(mm);
    __syncthreads();
    // exclusive prefix over warps per digit
    int acc = 0;
    for (int k = 0; k < WPB; k++) {
      const int v = wc[k][threadIdx.x];
      wc[k][threadIdx.x] = acc;
      acc += v;
    }
    __syncthreads();
    if (ok) {
      const int pos = run[dg] + wc[w][dg] + rank;
      key2[pos] = kk;
      val2[pos] = val[e];
    }
    __syncthreads();
    run[threadIdx.x] += acc;
    __syncthreads();
  }
}

// ---- prefix sums over sorted breakpoints ------------------------------------------
// For sorted breakpoint e (b = val[e], t_e, d_b, w_b): u = d_b w_b, v = t_e d_b w_b, s = d_b^2.
// Pass 1: sums per warp chunk. Layout of a partial: [u(0..col2) | v(0..col2) | s].
__global__ void k_gcp_sum(const unsigned long long* key, const int* val, int K, int chunk, const double* d,
                          const double* S, const double* Y, long long n, Cols c, double theta, double* part) {
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * NT + threadIdx.x) >> 5;
  const int col2 = 2 * c.col;
  const long long e0 = (long long)wg * chunk, e1 = min((long long)K, e0 + chunk);
  if (e0 >= e1) return;  // warps past the last chunk
  double u = 0.0, v = 0.0, s = 0.0;
  for (long long e = e0; e < e1; e++) {
    const int b = val[e];
    const double te = __longlong_as_double((long long)key[e]);
    const double db = d[b];
    const double w = lane < col2 ? wcol(S, Y, n, c, theta, lane, b) : 0.0;
    u += db * w;
    v += te * db * w;
    s += db * db;
  }
  const int nv = 2 * col2 + 1;
  if (lane < col2) {
    part[(long long)wg * nv + lane] = u;
    part[(long long)wg * nv + col2 + lane] = v;
  }
  if (lane == 0) part[(long long)wg * nv + 2 * col2] = s;
}

// Pass 2: exclusive prefix over warps of every component (fixed order)
__global__ void k_gcp_scan(double* part, int nw, int nv) {
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    double run = 0.0;
    for (int w = 0; w < nw; w++) {
      const double x = part[(long long)w * nv + k];
      part[(long long)w * nv + k] = run;
      run += x;
    }
  }
}

struct GcpScal {
  double theta, D2, f2org;
  int K;
};
// Pass 3: walk each chunk with running prefixes Q (sum d_b w_b), R (sum t d_b w_b), S2;
// after breakpoint j (1-based): P_j = p0 - Q_j, c_j = t_j P_{j-1} + R_{j-1},
// f' = -|d_j|^2 + theta t_j |d_j|^2 - c_j^T M P_j, f'' = theta |d_j|^2 - P_j^T M P_j.
// The first j with -f'/f'' < t_{j+1} - t_j (or j = K) holds the Cauchy point.
// cand[warp] = {j, dtm, t_j, P_j (col2), c_j (col2)}.
__global__ void k_gcp_search(const unsigned long long* key, const int* val, int chunk, const double* d,
                             const double* S, const double* Y, long long n, Cols c, GcpScal q, const double* part,
                             const double* p0, const double* Mmat, int* jstar, double* cand) {
  __shared__ double Ms[2 * MAXM][2 * MAXM];
  const int col2 = 2 * c.col;
  for (int k = threadIdx.x; k < col2 * col2; k += NT) Ms[k / col2][k % col2] = Mmat[k];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * NT + threadIdx.x) >> 5;
  const int nv = 2 * col2 + 1;
  const long long e0 = (long long)wg * chunk, e1 = min((long long)q.K, e0 + chunk);
  if (e0 >= e1) return;
  double Q = lane < col2 ? part[(long long)wg * nv + lane] : 0.0;
  double R = lane < col2 ? part[(long long)wg * nv + col2 + lane] : 0.0;
  double S2 = part[(long long)wg * nv + 2 * col2];
  const double p0l = lane < col2 ? p0[lane] : 0.0;
  for (long long e = e0; e < e1; e++) {
    if ((e & 63) == 0) {  // an earlier segment already holds the Cauchy point (warp-uniform test)
      int js = 0;
      if (lane == 0) js = *((volatile int*)jstar);
      js = __shfl_sync(0xffffffffu, js, 0);
      if (js <= e) return;
    }
    const int b = val[e];
    const double te = __longlong_as_double((long long)key[e]);
    const double db = d[b];
    const double w = lane < col2 ? wcol(S, Y, n, c, q.theta, lane, b) : 0.0;
    const double Cj = te * (p0l - Q) + R;  // c_j from P_{j-1}, R_{j-1}
    Q += db * w;
    R += te * db * w;
    S2 += db * db;
    const double Pj = p0l - Q;
    const double Dj = q.D2 - S2;
    double mp = 0.0;
    for (int a = 0; a < col2; a++) {
      const double pa = __shfl_sync(0xffffffffu, Pj, a);
      if (lane < col2) mp += Ms[lane][a] * pa;
    }
    double cmp = Cj * mp, pmp = Pj * mp;
    for (int o = 16; o; o >>= 1) {
      cmp += __shfl_xor_sync(0xffffffffu, cmp, o);
      pmp += __shfl_xor_sync(0xffffffffu, pmp, o);
    }
    const long long j = e + 1;
    double f1 = -Dj + q.theta * te * Dj - cmp;
    double f2 = fmax(EPSMCH * q.f2org, q.theta * Dj - pmp);
    double dtm;
    bool stop;
    if (j == q.K) {
      dtm = 0.0;  // every breakpoint passed: all moving variables at their bounds
      stop = true;
    } else {
      dtm = -f1 / f2;
      const double tn = __longlong_as_double((long long)key[e + 1]);
      stop = dtm < tn - te;
    }
    if (stop) {
      double* o = cand + (long long)wg * (3 + 2 * 2 * MAXM);
      if (lane == 0) {
        o[0] = (double)j;
        o[1] = dtm;
        o[2] = te;
        atomicMin(jstar, (int)j);
      }
      if (lane < col2) {
        o[3 + lane] = Pj;
        o[3 + col2 + lane] = Cj;
      }
      return;
    }
  }
}

// the winning warp's candidate {j, dtm, t_j, P_j, c_j} into out (one thread)
__global__ void k_pick_cand(const int* jstar, int chunk, const double* cand, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int js = *jstar;
  constexpr int cl = 3 + 2 * 2 * MAXM;
  if (js < 1 || js == 0x7fffffff) {
    out[0] = -1.0;
    return;
  }
  const double* c = cand + (long long)((js - 1) / chunk) * cl;
  for (int i = 0; i < cl; i++) out[i] = c[i];
}

// xcp = x + tsum d; free = moving or zero-gradient; then the first jst sorted
// breakpoints go to their bounds and leave the free set
__global__ void k_xcp(const double* x, const double* d, const int8_t* st, long long n, double tsum, double* xcp,
                      int8_t* fr) {
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    xcp[i] = x[i] + tsum * d[i];
    fr[i] = (st[i] == 0 || st[i] == 3) ? 1 : 0;
  }
}
__global__ void k_xcp_fix(const int* val, int jst, const double* d, double lo, double hi, double* xcp, int8_t* fr) {
  for (long long e = blockIdx.x * (long long)NT + threadIdx.x; e < jst; e += (long long)gridDim.x * NT) {
    const int b = val[e];
    xcp[b] = d[b] > 0.0 ? hi : lo;
    fr[b] = 0;
  }
}

// ---- subspace minimisation -----------------------------------------------------------
// r = -theta (xcp - x) - g + W (M c) on free variables (the negative reduced gradient)
__global__ void k_rgrad(const double* x, const double* g, const double* xcp, const int8_t* fr, long long n,
                        const double* S, const double* Y, Cols c, double theta, const double* Mc, double* r) {
  __shared__ double mc[2 * MAXM];
  const int col2 = 2 * c.col;
  if (threadIdx.x < col2) mc[threadIdx.x] = Mc[threadIdx.x];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    double ri = 0.0;
    if (fr[i]) {
      ri = -theta * (xcp[i] - x[i]) - g[i];
      for (int a = 0; a < col2; a++) ri += wcol(S, Y, n, c, theta, a, i) * mc[a];
    }
    r[i] = ri;
  }
}

// Gram of the unscaled columns [Y | S] over free variables, their products with r, and
// the number of free variables: partial layout [pairs (a <= b) | col2 | 1]
constexpr int GT = 64;
__global__ void k_gram(const int8_t* fr, const double* r, long long n, const double* S, const double* Y, Cols c,
                       double* part) {
  __shared__ double sh[2 * MAXM + 1][GT + 1];
  __shared__ unsigned char pa[2 * MAXM * (2 * MAXM + 1) / 2], pb[2 * MAXM * (2 * MAXM + 1) / 2];
  const int col2 = 2 * c.col;
  const int np = col2 * (col2 + 1) / 2, ntot = np + col2 + 1;
  if (threadIdx.x == 0) {
    int k = 0;
    for (int a = 0; a < col2; a++)
      for (int b = a; b < col2; b++) {
        pa[k] = (unsigned char)a;
        pb[k] = (unsigned char)b;
        k++;
      }
  }
  double acc[3] = {0.0, 0.0, 0.0};  // ntot <= 561 <= 3 * NT
  for (long long t0 = (long long)blockIdx.x * GT; t0 < n; t0 += (long long)gridDim.x * GT) {
    __syncthreads();
    for (int k = threadIdx.x; k < (col2 + 1) * GT; k += NT) {
      const int a = k / GT, e = k % GT;
      const long long i = t0 + e;
      double v = 0.0;
      if (i < n && fr[i]) {
        if (a < col2)
          v = a < c.col ? Y[(long long)c.slot[a] * n + i] : S[(long long)c.slot[a - c.col] * n + i];
        else
          v = r[i];
      }
      sh[a][e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 3; u++) {
      const int p = threadIdx.x + u * NT;
      if (p < np) {
        const int a = pa[p], b = pb[p];
        double s = 0.0;
        for (int e = 0; e < GT; e++) s += sh[a][e] * sh[b][e];
        acc[u] += s;
      } else if (p < np + col2) {
        const int a = p - np;
        double s = 0.0;
        for (int e = 0; e < GT; e++) s += sh[a][e] * sh[col2][e];
        acc[u] += s;
      } else if (p == np + col2) {
        double s = 0.0;
        for (int e = 0; e < GT; e++) {
          const long long i = t0 + e;
          s += (i < n && fr[i]) ? 1.0 : 0.0;
        }
        acc[u] += s;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 3; u++) {
    const int p = threadIdx.x + u * NT;
    if (p < ntot) part[(long long)blockIdx.x * ntot + p] = acc[u];
  }
}

// du = r / theta + (W v) / theta^2 on free variables; xbar = P(xcp + du) there, xcp elsewhere.
// sums: [0] (xbar - x) . g, [1] number of free variables that landed on a bound
__global__ void k_newton(const double* x, const double* g, const double* xcp, const int8_t* fr, long long n,
                         double lo, double hi, const double* S, const double* Y, Cols c, double theta,
                         const double* vv, double* r, double* xbar, double* part) {
  __shared__ double v[2 * MAXM];
  const int col2 = 2 * c.col;
  if (threadIdx.x < col2) v[threadIdx.x] = vv[threadIdx.x];
  __syncthreads();
  double s[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    double xb = xcp[i];
    if (fr[i]) {
      double wv = 0.0;
      for (int a = 0; a < col2; a++) wv += wcol(S, Y, n, c, theta, a, i) * v[a];
      const double du = r[i] / theta + wv / (theta * theta);
      r[i] = du;
      xb = fmin(hi, fmax(lo, xb + du));
      if (xb == lo || xb == hi) s[1] += 1.0;
    }
    xbar[i] = xb;
    s[0] += (xb - x[i]) * g[i];
  }
  block_sums<2>(s, 2, part);
}

// largest alpha <= 1 with xcp + alpha du feasible on free variables (first blocking index)
__global__ void k_alpha(const double* xcp, const double* du, const int8_t* fr, long long n, double lo, double hi,
                        VI* part) {
  VI m{1.0, -1};
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    if (!fr[i]) continue;
    const double dk = du[i];
    double tmp = 2.0;
    if (dk < 0.0) {
      const double t2 = lo - xcp[i];
      tmp = t2 >= 0.0 ? 0.0 : (dk < t2 ? t2 / dk : 2.0);
    } else if (dk > 0.0) {
      const double t2 = hi - xcp[i];
      tmp = t2 <= 0.0 ? 0.0 : (dk > t2 ? t2 / dk : 2.0);
    }
    if (tmp < 1.0) m = vimin(m, VI{tmp, i});
  }
  block_min(m, part);
}
__global__ void k_xbar_bt(const double* xcp, const double* du, const int8_t* fr, long long n, double alpha,
                          long long ibd, double lo, double hi, double* xbar) {
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    double xb = xcp[i];
    if (fr[i]) xb = (i == ibd) ? (du[i] > 0.0 ? hi : lo) : xb + alpha * du[i];
    xbar[i] = xb;
  }
}

// ---- line search ------------------------------------------------------------------
// d = xbar - x; sums [0] g.d, [1] d.d; min: the largest feasible step along d
__global__ void k_dir(const double* x, const double* g, const double* xbar, long long n, double lo, double hi,
                      double* d, double* part, VI* mpart) {
  double s[2] = {0.0, 0.0};
  VI m{BIG, -1};
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    const double di = xbar[i] - x[i];
    d[i] = di;
    s[0] += g[i] * di;
    s[1] += di * di;
    if (di < 0.0) {
      const double a2 = lo - x[i];
      m = vimin(m, VI{a2 >= 0.0 ? 0.0 : a2 / di, i});
    } else if (di > 0.0) {
      const double a2 = hi - x[i];
      m = vimin(m, VI{a2 <= 0.0 ? 0.0 : a2 / di, i});
    }
  }
  block_sums<2>(s, 2, part);
  block_min(m, mpart);
}

__global__ void k_trial(const double* x, const double* d, const double* xbar, long long n, double stp, double* xt,
                        float* e32, double* e64) {
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    const double v = stp == 1.0 ? xbar[i] : x[i] + stp * d[i];
    xt[i] = v;
    if (e32) e32[i] = (float)v;
    if (e64) e64[i] = v;
  }
}

// accepted step: optionally store s = stp d, y = gt - g in a slot; x = xt, g = gt.
// sums: [0] y.y, [1..col) s.Y_k, [col..2col) S_k.s over the retained pairs (before this one)
__global__ void k_accept(double* x, double* g, const double* xt, const double* gt, const double* d, long long n,
                         double stp, int store, double* Snew, double* Ynew, const double* S, const double* Y,
                         Cols c, double* part) {
  double v[2 * MAXM + 1];
#pragma unroll
  for (int k = 0; k < 2 * MAXM + 1; k++) v[k] = 0.0;
  for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
    const double si = stp * d[i], yi = gt[i] - g[i];
    if (store) {
      Snew[i] = si;
      Ynew[i] = yi;
      v[0] += yi * yi;
#pragma unroll
      for (int k = 0; k < MAXM; k++)
        if (k < c.col) {
          v[1 + k] += si * Y[(long long)c.slot[k] * n + i];
          v[1 + MAXM + k] += S[(long long)c.slot[k] * n + i] * si;
        }
    }
    x[i] = xt[i];
    g[i] = gt[i];
  }
  // pack [y.y | s.Y (col) | S.s (col)]
  double w[2 * MAXM + 1];
#pragma unroll
  for (int k = 0; k < 2 * MAXM + 1; k++) w[k] = 0.0;
  w[0] = v[0];
#pragma unroll
  for (int k = 0; k < MAXM; k++)
    if (k < c.col) {
      w[1 + k] = v[1 + k];
      w[1 + c.col + k] = v[1 + MAXM + k];
    }
  block_sums<2 * MAXM + 1>(w, 1 + 2 * c.col, part);
}

// ---- host: small dense linear algebra (Gauss-Jordan with partial pivoting) ---------------
bool solve_inplace(std::vector<double>& A, std::vector<double>& B, int n, int nrhs) {
  for (int k = 0; k < n; k++) {
    int p = k;
    for (int i = k + 1; i < n; i++)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; j++) std::swap(A[k * n + j], A[p * n + j]);
      for (int j = 0; j < nrhs; j++) std::swap(B[k * nrhs + j], B[p * nrhs + j]);
    }
    const double piv = A[k * n + k];
    for (int i = 0; i < n; i++) {
      if (i == k) continue;
      const double f = A[i * n + k] / piv;
      if (f == 0.0) continue;
      for (int j = k; j < n; j++) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < nrhs; j++) B[i * nrhs + j] -= f * B[k * nrhs + j];
    }
  }
  for (int i = 0; i < n; i++)
    for (int j = 0; j < nrhs; j++) B[i * nrhs + j] /= A[i * n + i];
  return true;
}

// ---- Line search of More and Thuente (ACM TOMS 20:286-307, 1994) ---------------------
// Looks for a step a > 0 along the direction with phi(a) = f(x + a d) satisfying the strong
// Wolfe conditions phi(a) <= phi(0) + mu a phi'(0) and |phi'(a)| <= eta |phi'(0)|, inside
// [amin, amax]. The paper's scheme: an interval of uncertainty [best, other] whose end
// "best" has the lowest value seen and a derivative that points into the interval; each
// trial step comes from cubic, quadratic and secant interpolation of the end points and
// the last trial (its four cases), safeguarded by a 0.66 shrink of bracketed steps, by
// bisection when two trials did not shrink the interval to 0.66 of its width, and by
// extrapolation limits [1.1, 4] times the last move while no minimiser is bracketed.
// Until a step with psi(a) = phi(a) - a mu phi'(0) - phi(0) <= 0 and phi'(a) >= 0 is
// seen (stage 1), trial values are taken on psi, afterwards on phi.
struct Probe {
  double a, f, g;  // step, value, derivative along d
};

// Minimiser of the cubic with values and slopes p and q at p.a and q.a (the same cubic,
// and so the same point, whichever end is p). With t = p.g + q.g - 3 (secant slope) the
// slope of the cubic has the roots p.a + h (t - p.g +- sqrt(t^2 - p.g q.g)) / (...);
// the minimiser takes the root whose sign follows h = q.a - p.a. Values are divided by
// the largest of |t|, |p.g|, |q.g| before squaring, so nothing overflows.
double cubic_min(const Probe& p, const Probe& q) {
  const double h = q.a - p.a;
  const double t = 3.0 * (p.f - q.f) / h + p.g + q.g;
  const double m = std::max(std::fabs(t), std::max(std::fabs(p.g), std::fabs(q.g)));
  const double disc = (t / m) * (t / m) - (p.g / m) * (q.g / m);
  const double root = (h > 0.0 ? 1.0 : -1.0) * m * std::sqrt(disc);
  const double r = ((root - p.g) + t) / (((root - p.g) + root) + q.g);
  return p.a + r * h;
}

// the same cubic in the form used where the minimiser is only accepted when it lies on
// the side of q away from p (stage 3): *valid is false when there is no such minimiser
double cubic_min_beyond(const Probe& p, const Probe& q, bool* valid) {
  const double h = p.a - q.a;
  const double t = 3.0 * (p.f - q.f) / (q.a - p.a) + p.g + q.g;
  const double m = std::max(std::fabs(t), std::max(std::fabs(p.g), std::fabs(q.g)));
  const double disc = std::max(0.0, (t / m) * (t / m) - (p.g / m) * (q.g / m));
  const double root = (q.a > p.a ? -1.0 : 1.0) * m * std::sqrt(disc);
  const double num = (root - q.g) + t, den = (root + (p.g - q.g)) + root;
  const double r = num / den;
  *valid = r < 0.0 && root != 0.0;
  return q.a + r * h;
}

// minimiser of the quadratic with value and slope p at p.a and value qf at qa
double quad_min(const Probe& p, double qa, double qf) {
  const double h = qa - p.a;
  return p.a + (p.g / ((p.f - qf) / h + p.g)) / 2.0 * h;
}

// zero of the straight line through the slopes of p and q
double secant_min(const Probe& p, const Probe& q) { return q.a + (q.g / (q.g - p.g)) * (p.a - q.a); }

class MoreThuente {
 public:
  double mu = 1e-3, eta = 0.9, xtol = 0.1;  // sufficient decrease, curvature, relative interval width
  double amin = 0.0, amax = 0.0;

  // phi(0) = f0, phi'(0) = g0 < 0, first trial a1
  void begin(double f0, double g0, double a1) {
    f0_ = f0;
    g0_ = g0;
    dec_ = mu * g0;
    bracketed_ = false;
    stage2_ = false;
    width_ = amax - amin;
    width_old_ = 2.0 * width_;
    best_ = {0.0, f0, g0};
    other_ = {0.0, f0, g0};
    lo_ = 0.0;
    hi_ = a1 + 4.0 * a1;
  }

  // phi(a) = f, phi'(a) = g at the trial a; true: accept a; false: a holds the next trial
  bool advance(double f, double g, double& a) {
    const double fsuff = f0_ + a * dec_;  // sufficient-decrease line
    if (!stage2_ && f <= fsuff && g >= 0.0) stage2_ = true;
    if (converged(f, g, a, fsuff)) return true;
    Probe t = {a, f, g};
    if (!stage2_ && f <= best_.f && f > fsuff) {
      // stage 1 on psi: shift every value and slope by the sufficient-decrease line
      Probe b = shifted(best_), o = shifted(other_), ts = shifted(t);
      a = trial(b, o, ts);
      best_ = unshifted(b);
      other_ = unshifted(o);
    } else {
      a = trial(best_, other_, t);
    }
    if (bracketed_) {
      const double w = std::fabs(other_.a - best_.a);
      if (w >= 0.66 * width_old_) a = best_.a + 0.5 * (other_.a - best_.a);  // bisection
      width_old_ = width_;
      width_ = w;
      lo_ = std::min(best_.a, other_.a);
      hi_ = std::max(best_.a, other_.a);
    } else {
      lo_ = a + 1.1 * (a - best_.a);
      hi_ = a + 4.0 * (a - best_.a);
    }
    a = std::min(std::max(a, amin), amax);
    // no progress possible within the interval: fall back to the best step
    if (bracketed_ && (a <= lo_ || a >= hi_ || hi_ - lo_ <= xtol * hi_)) a = best_.a;
    return false;
  }

 private:
  double f0_ = 0, g0_ = 0, dec_ = 0, width_ = 0, width_old_ = 0, lo_ = 0, hi_ = 0;
  bool bracketed_ = false, stage2_ = false;
  Probe best_{}, other_{};

  Probe shifted(const Probe& p) const { return {p.a, p.f - p.a * dec_, p.g - dec_}; }
  Probe unshifted(const Probe& p) const { return {p.a, p.f + p.a * dec_, p.g + dec_}; }

  bool converged(double f, double g, double a, double fsuff) const {
    if (bracketed_ && (a <= lo_ || a >= hi_)) return true;          // rounding stops progress
    if (bracketed_ && hi_ - lo_ <= xtol * hi_) return true;         // interval below tolerance
    if (a == amax && f <= fsuff && g <= dec_) return true;          // at the upper bound
    if (a == amin && (f > fsuff || g >= dec_)) return true;         // at the lower bound
    return f <= fsuff && std::fabs(g) <= eta * (-g0_);              // strong Wolfe conditions
  }

  // Next trial from the interval ends b (best), o (other) and the trial t (the paper's four
  // cases), then the interval update: t replaces o when its value is higher than b's;
  // otherwise t becomes the best end, and o moves to the old best when the slopes of b
  // and t have opposite signs.
  double trial(Probe& b, Probe& o, const Probe& t) {
    const bool opposite = t.g * (b.g / std::fabs(b.g)) < 0.0;
    double next;
    if (t.f > b.f) {  // case 1: higher value, a minimiser lies between b and t
      const double c = cubic_min(b, t);
      const double q = quad_min(b, t.a, t.f);
      next = std::fabs(c - b.a) < std::fabs(q - b.a) ? c : c + (q - c) / 2.0;
      bracketed_ = true;
    } else if (opposite) {  // case 2: lower value, slopes of opposite signs
      const double c = cubic_min(b, t);
      const double sc = secant_min(b, t);
      next = std::fabs(c - t.a) > std::fabs(sc - t.a) ? c : sc;
      bracketed_ = true;
    } else if (std::fabs(t.g) < std::fabs(b.g)) {  // case 3: lower value, slope shrinking
      bool valid = false;
      double c = cubic_min_beyond(b, t, &valid);
      if (!valid) c = t.a > b.a ? hi_ : lo_;
      const double sc = secant_min(b, t);
      if (bracketed_) {
        next = std::fabs(c - t.a) < std::fabs(sc - t.a) ? c : sc;
        const double lim = t.a + 0.66 * (o.a - t.a);
        next = t.a > b.a ? std::min(lim, next) : std::max(lim, next);
      } else {
        next = std::fabs(c - t.a) > std::fabs(sc - t.a) ? c : sc;
        next = std::max(lo_, std::min(hi_, next));
      }
    } else {  // case 4: lower value, slope not shrinking
      next = bracketed_ ? cubic_min(o, t) : (t.a > b.a ? hi_ : lo_);
    }
    if (t.f > b.f) {
      o = t;
    } else {
      if (opposite) o = b;
      b = t;
    }
    return next;
  }
};

int grid_for(long long n, int nsm) {
  const long long b = (n + NT - 1) / NT;
  return (int)std::max(1LL, std::min(b, 4LL * nsm));
}

}  // namespace

struct tm_lbfgsb {
  int device = 0, nsm = 148;
  long long n = 0;
  int m = 10, maxls = 20;
  double lo = 0, hi = 1, factr = 1e7, pgtol = 1e-5;
  std::string err;
  // device state
  double *x = nullptr, *g = nullptr, *xt = nullptr, *gt = nullptr, *d = nullptr, *xcp = nullptr, *xbar = nullptr,
         *r = nullptr, *t = nullptr, *S = nullptr, *Y = nullptr;
  int8_t *st = nullptr, *fr = nullptr;
  unsigned long long *key = nullptr, *key2 = nullptr;
  int *val = nullptr, *val2 = nullptr, *cnt = nullptr, *hist = nullptr, *jstar = nullptr;
  double *part = nullptr, *red = nullptr, *small = nullptr, *cand = nullptr;
  VI *mpart = nullptr, *mred = nullptr;
  size_t part_doubles = 0;
  double* hbuf = nullptr;  // pinned
  // host state
  int col = 0, head = 0;               // pairs in memory, slot of the oldest
  std::vector<double> SY, SS;          // logical order, MAXM x MAXM (SY lower, SS upper)
  double theta = 1.0, f = 0.0, fold = 0.0, sbgnrm = 0.0;
  long long iter = 0, nfev = 0, nbreak = 0, nfree = 0;
  int phase = 0;  // 0 created, 1 waiting for f(x0), 2 in a line search, 3 new x reported, 4 stopped
  // line search state
  MoreThuente ls;
  double stp = 1.0, gd = 0.0, dtd = 0.0, stpmx = 0.0;
  int nls = 0;
};

namespace {

int fail(tm_lbfgsb* o, int code, const std::string& msg) {
  if (o) o->err = msg;
  return code;
}
#define LCK(call)                                                               \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) return fail(o, TM_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)
#define LCKL() LCK(cudaGetLastError())

Cols cols_of(const tm_lbfgsb* o) {
  Cols c;
  c.col = o->col;
  for (int k = 0; k < MAXM; k++) c.slot[k] = k < o->col ? (o->head + k) % o->m : 0;
  return c;
}

// sums in o->part (nblk partials of nv) -> host hbuf[0..nv)
int fetch_sums(tm_lbfgsb* o, int nblk, int nv, cudaStream_t s) {
  k_finish<<<1, 256, 0, s>>>(o->part, nblk, nv, o->red);
  LCKL();
  LCK(cudaMemcpyAsync(o->hbuf, o->red, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  LCK(cudaStreamSynchronize(s));
  return TM_OK;
}
// sums (nblk_s partials of nv) to hbuf[0..nv) and the min of nblk_m partials to *out, one sync
int fetch_both(tm_lbfgsb* o, int nblk_s, int nv, int nblk_m, VI* out, cudaStream_t s) {
  k_finish<<<1, 256, 0, s>>>(o->part, nblk_s, nv, o->red);
  LCKL();
  k_finish_min<<<1, 32, 0, s>>>(o->mpart, nblk_m, o->mred);
  LCKL();
  LCK(cudaMemcpyAsync(o->hbuf, o->red, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  LCK(cudaMemcpyAsync(out, o->mred, sizeof(VI), cudaMemcpyDeviceToHost, s));
  LCK(cudaStreamSynchronize(s));
  return TM_OK;
}
int fetch_min(tm_lbfgsb* o, int nblk, VI* out, cudaStream_t s) {
  k_finish_min<<<1, 32, 0, s>>>(o->mpart, nblk, o->mred);
  LCKL();
  LCK(cudaMemcpyAsync(out, o->mred, sizeof(VI), cudaMemcpyDeviceToHost, s));
  LCK(cudaStreamSynchronize(s));
  return TM_OK;
}

// the inverse middle matrix [[-D, L^T], [L, theta S^T S]] (2col x 2col, row-major)
std::vector<double> middle_inv(const tm_lbfgsb* o) {
  const int c = o->col, c2 = 2 * c;
  std::vector<double> K(c2 * c2, 0.0);
  for (int i = 0; i < c; i++)
    for (int j = 0; j < c; j++) {
      if (i == j) K[i * c2 + j] = -o->SY[i * MAXM + i];
      if (i > j) {  // L_ij = s_i . y_j
        K[(c + i) * c2 + j] = o->SY[i * MAXM + j];
        K[j * c2 + (c + i)] = o->SY[i * MAXM + j];
      }
      const double ss = i <= j ? o->SS[i * MAXM + j] : o->SS[j * MAXM + i];
      K[(c + i) * c2 + (c + j)] = o->theta * ss;
    }
  return K;
}

// Cauchy point and subspace step from (x, g): fills xbar. Returns TM_OK or an error.
int direction(tm_lbfgsb* o, cudaStream_t s) {
  const long long n = o->n;
  const Cols c = cols_of(o);
  const int col2 = 2 * o->col;
  const double theta = o->theta;
  const int ntile = (int)((n + TILE - 1) / TILE);
  // breakpoints, p0 = W^T d, d.d
  k_bp<<<ntile, NT, 0, s>>>(o->x, o->g, n, o->lo, o->hi, o->S, o->Y, c, theta, o->d, o->t, o->st, o->part, o->cnt,
                            o->mpart);
  LCKL();
  k_scan_ex<<<1, 1024, 0, s>>>(o->cnt, ntile);
  LCKL();
  int* Kh = reinterpret_cast<int*>(o->hbuf + 1000);  // pinned slot for the count
  LCK(cudaMemcpyAsync(Kh, o->cnt + ntile, sizeof(int), cudaMemcpyDeviceToHost, s));
  VI tmin;
  if (int e = fetch_both(o, ntile, col2 + 1, ntile, &tmin, s)) return e;
  std::vector<double> p0(o->hbuf, o->hbuf + col2);
  const double D2 = o->hbuf[col2];
  const int K = *Kh;
  o->nbreak = K;
  std::vector<double> Minv, M;
  if (o->col > 0) {
    Minv = middle_inv(o);
    std::vector<double> A = Minv;
    M.assign(col2 * col2, 0.0);
    for (int i = 0; i < col2; i++) M[i * col2 + i] = 1.0;
    if (!solve_inplace(A, M, col2, col2)) return fail(o, TM_ERR_STATE, "singular limited-memory matrix");
  }
  double tsum = 0.0;
  std::vector<double> cvec(col2, 0.0);
  int jst = 0;
  if (D2 == 0.0) {  // no variable moves: the Cauchy point is x
    tsum = 0.0;
  } else {
    double pmp = 0.0;
    for (int a = 0; a < col2; a++)
      for (int b = 0; b < col2; b++) pmp += p0[a] * M[a * col2 + b] * p0[b];
    const double f1 = -D2, f2org = theta * D2, f2 = f2org - pmp;
    const double dtm0 = -f1 / f2;
    // the smallest breakpoint decides whether the minimiser lies before it; only then
    // is the sort (and the breakpoint scan) needed
    const double t1 = K > 0 ? tmin.v : INFINITY;
    if (K > 0 && !(dtm0 < t1)) {
      k_bp_compact<<<ntile, NT, 0, s>>>(o->t, o->st, n, o->cnt, o->key, o->val);
      LCKL();
      // sort by t (stable, so equal t keep index order)
      const int kt = (K + TILE - 1) / TILE;
      unsigned long long *k1 = o->key, *k2 = o->key2;
      int *v1 = o->val, *v2 = o->val2;
      for (int sh = 0; sh < 64; sh += 8) {
        k_rs_hist<<<kt, NT, 0, s>>>(k1, K, sh, o->hist, kt);
        LCKL();
        k_scan_ex<<<1, 1024, 0, s>>>(o->hist, 256LL * kt);
        LCKL();
        k_rs_scatter<<<kt, NT, 0, s>>>(k1, v1, K, sh, o->hist, kt, k2, v2);
        LCKL();
        std::swap(k1, k2);
        std::swap(v1, v2);
      }
    }
    if (K == 0 || dtm0 < t1) {
      jst = 0;
      const double dtm = std::max(dtm0, 0.0);
      tsum = dtm;
      for (int a = 0; a < col2; a++) cvec[a] = dtm * p0[a];
    } else {
      const int nw = std::min(WPB * 4 * o->nsm, K);
      const int chunk = (K + nw - 1) / nw;
      const int nwu = (K + chunk - 1) / chunk;
      const int blocks = (nwu + WPB - 1) / WPB;
      k_gcp_sum<<<blocks, NT, 0, s>>>(o->key, o->val, K, chunk, o->d, o->S, o->Y, n, c, theta, o->part);
      LCKL();
      k_gcp_scan<<<1, 128, 0, s>>>(o->part, nwu, 2 * col2 + 1);
      LCKL();
      // small: p0 (col2), M (col2^2)
      std::vector<double> hs(col2 + col2 * col2);
      std::copy(p0.begin(), p0.end(), hs.begin());
      std::copy(M.begin(), M.end(), hs.begin() + col2);
      if (!hs.empty()) LCK(cudaMemcpyAsync(o->small, hs.data(), hs.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      const int big = 0x7fffffff;
      LCK(cudaMemcpyAsync(o->jstar, &big, sizeof(int), cudaMemcpyHostToDevice, s));
      GcpScal q{theta, D2, f2org, K};
      k_gcp_search<<<blocks, NT, 0, s>>>(o->key, o->val, chunk, o->d, o->S, o->Y, n, c, q, o->part, o->small,
                                        o->small + col2, o->jstar, o->cand);
      LCKL();
      const int cl = 3 + 2 * 2 * MAXM;
      k_pick_cand<<<1, 32, 0, s>>>(o->jstar, chunk, o->cand, o->red);
      LCKL();
      LCK(cudaMemcpyAsync(o->hbuf, o->red, cl * sizeof(double), cudaMemcpyDeviceToHost, s));
      LCK(cudaStreamSynchronize(s));
      const int js = (int)o->hbuf[0];
      if (js < 1 || js > K) return fail(o, TM_ERR_STATE, "Cauchy point search found no segment");
      jst = js;
      const double dtm = std::max(o->hbuf[1], 0.0);
      tsum = o->hbuf[2] + dtm;
      for (int a = 0; a < col2; a++) cvec[a] = o->hbuf[3 + col2 + a] + dtm * o->hbuf[3 + a];
    }
  }
  const int gb = grid_for(n, o->nsm);
  k_xcp<<<gb, NT, 0, s>>>(o->x, o->d, o->st, n, tsum, o->xcp, o->fr);
  LCKL();
  if (jst > 0) {
    k_xcp_fix<<<grid_for(jst, o->nsm), NT, 0, s>>>(o->val, jst, o->d, o->lo, o->hi, o->xcp, o->fr);
    LCKL();
  }
  // subspace minimisation on the free variables
  if (o->col == 0) {
    LCK(cudaMemcpyAsync(o->xbar, o->xcp, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    o->nfree = -1;
    return TM_OK;
  }
  std::vector<double> Mc(col2, 0.0);
  for (int a = 0; a < col2; a++)
    for (int b = 0; b < col2; b++) Mc[a] += M[a * col2 + b] * cvec[b];
  LCK(cudaMemcpyAsync(o->small, Mc.data(), col2 * sizeof(double), cudaMemcpyHostToDevice, s));
  k_rgrad<<<gb, NT, 0, s>>>(o->x, o->g, o->xcp, o->fr, n, o->S, o->Y, c, theta, o->small, o->r);
  LCKL();
  const int np = col2 * (col2 + 1) / 2, ntot = np + col2 + 1;
  const int gg = std::max(1, std::min((int)((n + GT - 1) / GT), 2 * o->nsm));
  k_gram<<<gg, NT, 0, s>>>(o->fr, o->r, n, o->S, o->Y, c, o->part);
  LCKL();
  if (int e = fetch_sums(o, gg, ntot, s)) return e;
  const double* h = o->hbuf;
  o->nfree = (long long)h[np + col2];
  if (o->nfree == 0) {
    LCK(cudaMemcpyAsync(o->xbar, o->xcp, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return TM_OK;
  }
  // K' = Minv - (1/theta) W_F^T W_F with W = [Y, theta S]; rhs = W_F^T r
  std::vector<double> A = Minv, rhs(col2);
  int k = 0;
  for (int a = 0; a < col2; a++)
    for (int b = a; b < col2; b++, k++) {
      const double sa = a < o->col ? 1.0 : theta, sb = b < o->col ? 1.0 : theta;
      const double v = h[k] * sa * sb / theta;
      A[a * col2 + b] -= v;
      if (a != b) A[b * col2 + a] -= v;
    }
  for (int a = 0; a < col2; a++) rhs[a] = h[np + a] * (a < o->col ? 1.0 : theta);
  if (!solve_inplace(A, rhs, col2, 1)) return fail(o, TM_ERR_STATE, "singular reduced system");
  LCK(cudaMemcpyAsync(o->small, rhs.data(), col2 * sizeof(double), cudaMemcpyHostToDevice, s));
  k_newton<<<gb, NT, 0, s>>>(o->x, o->g, o->xcp, o->fr, n, o->lo, o->hi, o->S, o->Y, c, theta, o->small, o->r,
                             o->xbar, o->part);
  LCKL();
  if (int e = fetch_sums(o, gb, 2, s)) return e;
  const double ddp = o->hbuf[0], hit = o->hbuf[1];
  if (hit > 0.0 && ddp > 0.0) {  // projected point is not a descent step: backtrack onto the box
    k_alpha<<<gb, NT, 0, s>>>(o->xcp, o->r, o->fr, n, o->lo, o->hi, o->mpart);
    LCKL();
    VI a;
    if (int e = fetch_min(o, gb, &a, s)) return e;
    const double alpha = std::min(1.0, a.v);
    k_xbar_bt<<<gb, NT, 0, s>>>(o->xcp, o->r, o->fr, n, alpha, alpha < 1.0 ? a.i : -1, o->lo, o->hi, o->xbar);
    LCKL();
  }
  return TM_OK;
}

// start the line search along d = xbar - x; writes the first trial point
int begin_search(tm_lbfgsb* o, float* e32, double* e64, cudaStream_t s, bool& ascent) {
  const long long n = o->n;
  const int gb = grid_for(n, o->nsm);
  k_dir<<<gb, NT, 0, s>>>(o->x, o->g, o->xbar, n, o->lo, o->hi, o->d, o->part, o->mpart);
  LCKL();
  VI m;
  if (int e = fetch_both(o, gb, 2, gb, &m, s)) return e;
  o->gd = o->hbuf[0];
  o->dtd = o->hbuf[1];
  o->stpmx = o->iter == 0 ? 1.0 : std::min(BIG, m.v);
  ascent = !(o->gd < 0.0);
  if (ascent) return TM_OK;
  o->stp = 1.0;  // every variable has both bounds
  o->ls.amin = 0.0;
  o->ls.amax = o->stpmx;
  o->ls.begin(o->f, o->gd, o->stp);
  o->nls = 0;
  k_trial<<<gb, NT, 0, s>>>(o->x, o->d, o->xbar, n, o->stp, o->xt, e32, e64);
  LCKL();
  o->nls = 1;
  o->phase = 2;
  return TM_OK;
}

// compute a direction from the current (x, g) and start its line search; on an ascent
// direction drop the memory and retry once, then stop
int new_iteration(tm_lbfgsb* o, float* e32, double* e64, int* task, cudaStream_t s) {
  for (int attempt = 0; attempt < 2; attempt++) {
    if (int e = direction(o, s)) return e;
    bool ascent = false;
    if (int e = begin_search(o, e32, e64, s, ascent)) return e;
    if (!ascent) {
      *task = TM_LB_FG;
      return TM_OK;
    }
    if (o->col == 0) break;
    o->col = 0;
    o->head = 0;
    o->theta = 1.0;
  }
  o->phase = 4;
  *task = TM_LB_ABNORMAL;
  return TM_OK;
}

}  // namespace

extern "C" {

int tm_lbfgsb_create(tm_lbfgsb** out, int device, long long n, int m, double lower, double upper, double factr,
                     double pgtol, int maxls) {
  if (!out || n < 1 || n > 2000000000LL || m < 1 || m > MAXM || !(lower < upper) || !(factr >= 0) ||
      !(pgtol >= 0) || maxls < 1)
    return TM_ERR_ARG;
  tm_lbfgsb* o = new tm_lbfgsb();
  o->device = device;
  o->n = n;
  o->m = m;
  o->lo = lower;
  o->hi = upper;
  o->factr = factr;
  o->pgtol = pgtol;
  o->maxls = maxls;
  o->SY.assign(MAXM * MAXM, 0.0);
  o->SS.assign(MAXM * MAXM, 0.0);
  *out = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&o->nsm, cudaDevAttrMultiProcessorCount, device);
  const long long ntile = (n + TILE - 1) / TILE;
  const long long nwmax = (long long)WPB * 4 * o->nsm;
  o->part_doubles = (size_t)std::max({ntile * (2 * MAXM + 1), nwmax * (4 * MAXM + 1), 4LL * o->nsm * 600,
                                      (long long)grid_for(n, o->nsm) * (2 * MAXM + 1)});
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  const size_t nd = (size_t)n * sizeof(double);
  A((void**)&o->x, nd);
  A((void**)&o->g, nd);
  A((void**)&o->xt, nd);
  A((void**)&o->gt, nd);
  A((void**)&o->d, nd);
  A((void**)&o->xcp, nd);
  A((void**)&o->xbar, nd);
  A((void**)&o->r, nd);
  A((void**)&o->t, nd);
  A((void**)&o->S, nd * m);
  A((void**)&o->Y, nd * m);
  A((void**)&o->st, n);
  A((void**)&o->fr, n);
  A((void**)&o->key, n * sizeof(unsigned long long));
  A((void**)&o->key2, n * sizeof(unsigned long long));
  A((void**)&o->val, n * sizeof(int));
  A((void**)&o->val2, n * sizeof(int));
  A((void**)&o->cnt, (ntile + 1) * sizeof(int));
  A((void**)&o->hist, (256 * ntile + 1) * sizeof(int));
  A((void**)&o->jstar, sizeof(int));
  A((void**)&o->part, o->part_doubles * sizeof(double));
  A((void**)&o->red, 1024 * sizeof(double));
  A((void**)&o->small, (2 * MAXM + 4 * MAXM * MAXM) * sizeof(double));
  A((void**)&o->cand, nwmax * (3 + 4 * MAXM) * sizeof(double));
  A((void**)&o->mpart, std::max(8LL * o->nsm, ntile) * sizeof(VI));  // also one per k_bp tile
  A((void**)&o->mred, sizeof(VI));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&o->hbuf, 1024 * sizeof(double));
  if (e != cudaSuccess) {
    tm_lbfgsb_destroy(o);
    return e == cudaErrorMemoryAllocation ? TM_ERR_NOMEM : TM_ERR_CUDA;
  }
  *out = o;
  return TM_OK;
}

void tm_lbfgsb_destroy(tm_lbfgsb* o) {
  if (!o) return;
  cudaSetDevice(o->device);
  void* ps[] = {o->x,   o->g,    o->xt,   o->gt,  o->d,    o->xcp,   o->xbar, o->r,     o->t,
                o->S,   o->Y,    o->st,   o->fr,  o->key,  o->key2,  o->val,  o->val2,  o->cnt,
                o->hist, o->jstar, o->part, o->red, o->small, o->cand, o->mpart, o->mred};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (o->hbuf) cudaFreeHost(o->hbuf);
  delete o;
}

const char* tm_lbfgsb_last_error(const tm_lbfgsb* o) { return o ? o->err.c_str() : "null handle"; }

int tm_lbfgsb_start(tm_lbfgsb* o, const float* x0_32, const double* x0_64, float* e32, double* e64, int* task,
                    void* stream) {
  if (!o || !task || (!x0_32 && !x0_64) || (!e32 && !e64)) return fail(o, TM_ERR_ARG, "null argument");
  LCK(cudaSetDevice(o->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_start<<<grid_for(o->n, o->nsm), NT, 0, s>>>(x0_32, x0_64, o->n, o->lo, o->hi, o->x, e32, e64);
  LCKL();
  o->col = 0;
  o->head = 0;
  o->theta = 1.0;
  o->iter = 0;
  o->nfev = 0;
  o->phase = 1;
  *task = TM_LB_FG;
  return TM_OK;
}

int tm_lbfgsb_iterate(tm_lbfgsb* o, double f, const float* g32, const double* g64, float* e32, double* e64,
                      int* task, void* stream) {
  if (!o || !task || (!e32 && !e64)) return fail(o, TM_ERR_ARG, "null argument");
  if (o->phase == 0 || o->phase == 4) return fail(o, TM_ERR_STATE, "not started, or already stopped");
  if ((o->phase == 1 || o->phase == 2) && ((!g32 && !g64) || !std::isfinite(f)))
    return fail(o, TM_ERR_ARG, "an evaluation needs a finite f and a gradient");
  LCK(cudaSetDevice(o->device));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long n = o->n;
  const int gb = grid_for(n, o->nsm);
  if (o->phase == 1) {  // f, g at x0
    o->nfev++;
    o->f = f;
    k_load_g<<<gb, NT, 0, s>>>(g32, g64, n, nullptr, o->g, o->part);
    LCKL();
    k_projgr<<<gb, NT, 0, s>>>(o->x, o->g, n, o->lo, o->hi, o->mpart);
    LCKL();
    VI m;
    if (int e = fetch_min(o, gb, &m, s)) return e;
    o->sbgnrm = -m.v;
    if (o->sbgnrm <= o->pgtol) {
      o->phase = 4;
      *task = TM_LB_CONV_PGTOL;
      return TM_OK;
    }
    return new_iteration(o, e32, e64, task, s);
  }
  if (o->phase == 3) return new_iteration(o, e32, e64, task, s);
  // phase 2: f, g at the trial point x + stp d
  o->nfev++;
  k_load_g<<<gb, NT, 0, s>>>(g32, g64, n, o->d, o->gt, o->part);
  LCKL();
  if (int e = fetch_sums(o, gb, 1, s)) return e;
  const double gdt = o->hbuf[0];
  double stp = o->stp;
  const bool accepted = o->ls.advance(f, gdt, stp);
  if (!accepted) {
    if (o->nls >= o->maxls) {  // too many trials: drop the memory and restart from x, or stop
      if (o->col == 0) {
        o->phase = 4;
        *task = TM_LB_ABNORMAL;
        return TM_OK;
      }
      o->col = 0;
      o->head = 0;
      o->theta = 1.0;
      return new_iteration(o, e32, e64, task, s);
    }
    o->stp = stp;
    k_trial<<<gb, NT, 0, s>>>(o->x, o->d, o->xbar, n, o->stp, o->xt, e32, e64);
    LCKL();
    o->nls++;
    *task = TM_LB_FG;
    return TM_OK;
  }
  // accept x + stp d
  o->iter++;
  const double dr = (gdt - o->gd) * o->stp;
  const double ddum = -o->gd * o->stp;
  const bool store = !(dr <= EPSMCH * ddum);
  int slot = 0;
  Cols c = cols_of(o);
  if (store) {
    if (o->col < o->m) {
      slot = (o->head + o->col) % o->m;
    } else {  // the oldest pair leaves
      slot = o->head;
      c.col = o->m - 1;
      for (int k = 0; k < c.col; k++) c.slot[k] = (o->head + 1 + k) % o->m;
    }
  }
  k_accept<<<gb, NT, 0, s>>>(o->x, o->g, o->xt, o->gt, o->d, n, o->stp, store ? 1 : 0, o->S + (long long)slot * n,
                             o->Y + (long long)slot * n, o->S, o->Y, c, o->part);
  LCKL();
  k_projgr<<<gb, NT, 0, s>>>(o->x, o->g, n, o->lo, o->hi, o->mpart);  // after the accepted x, g
  LCKL();
  VI m;
  if (int e = fetch_both(o, gb, 1 + 2 * c.col, gb, &m, s)) return e;
  std::vector<double> h(o->hbuf, o->hbuf + 1 + 2 * c.col);
  o->fold = o->f;
  o->f = f;
  o->sbgnrm = -m.v;
  if (store) {
    if (o->col == o->m) {  // shift the retained pairs' products up-left
      for (int i = 0; i < o->m - 1; i++)
        for (int j = 0; j < o->m - 1; j++) {
          o->SY[i * MAXM + j] = o->SY[(i + 1) * MAXM + (j + 1)];
          o->SS[i * MAXM + j] = o->SS[(i + 1) * MAXM + (j + 1)];
        }
      o->head = (o->head + 1) % o->m;
    } else {
      o->col++;
    }
    const int nw = o->col - 1;  // logical index of the new pair
    for (int j = 0; j < nw; j++) {
      o->SY[nw * MAXM + j] = h[1 + j];        // s_new . y_j
      o->SS[j * MAXM + nw] = h[1 + c.col + j];  // s_j . s_new
    }
    o->SS[nw * MAXM + nw] = o->stp * o->stp * o->dtd;
    o->SY[nw * MAXM + nw] = dr;
    o->theta = h[0] / dr;
  }
  if (o->sbgnrm <= o->pgtol) {
    o->phase = 4;
    *task = TM_LB_CONV_PGTOL;
    return TM_OK;
  }
  if (o->fold - o->f <= o->factr * EPSMCH * std::max(std::fabs(o->fold), std::max(std::fabs(o->f), 1.0))) {
    o->phase = 4;
    *task = TM_LB_CONV_REL_F;
    return TM_OK;
  }
  // report the new iterate
  k_trial<<<gb, NT, 0, s>>>(o->x, o->d, o->x, n, 1.0, o->xt, e32, e64);
  LCKL();
  o->phase = 3;
  *task = TM_LB_NEW_X;
  return TM_OK;
}

int tm_lbfgsb_info(const tm_lbfgsb* o, long long counts[5], double values[3]) {
  if (!o || !counts || !values) return TM_ERR_ARG;
  counts[0] = o->iter;
  counts[1] = o->nfev;
  counts[2] = o->col;
  counts[3] = o->nbreak;
  counts[4] = o->nfree;
  values[0] = o->f;
  values[1] = o->sbgnrm;
  values[2] = o->theta;
  return TM_OK;
}

}  // extern "C"
