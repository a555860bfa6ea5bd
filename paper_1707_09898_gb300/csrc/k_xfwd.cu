// Forward x pass of the stray-field convolution (Sec. "Discretization", Eq. (convolution)).
//
// Real rows (rho^p, rho^p M0_c of Sec. "Methodology" Eq. 2, or a given vector
// component) are zero padded from nx to L (the first DIF stage reads only x < nx) and
// transformed two rows at a time (row a + i row b), then separated into the half
// spectra kx = 0..L/2. The first stage maps consecutive threads to consecutive x of
// one row pair, so global rows are read in 64-byte runs straight into registers; the
// half-spectrum rows are written with consecutive threads on consecutive kx.
#include "tma.cuh"
#include "xpass.cuh"

namespace tmk {

namespace {

__device__ __forceinline__ void cp16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp4(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Persistent: a block loops over 32-row tiles; the raw inputs of the next tile are
// loaded into registers while the current tile is separated and stored, so global
// latency overlaps the shared-memory work. P3: p = 3 fixed at compile time. UPD: the
// pending projected-gradient step of the previous iteration (Sec. "Methodology", box
// constraint) is applied to each rho value as it is used, and the new rho written back,
// with the arithmetic of the stand-alone update kernel (same results bit for bit).
template <int L, int SRC, bool P3, bool UPD>
__global__ void __launch_bounds__(kNT, 2) k_xfwd(XFwdArgs a) {
  constexpr int S = plan_stages(L);
  using S0 = StageShape<L, 0>;
  constexpr bool withM0 = SRC == SRC_RHO_M0;
  constexpr int RM = withM0 ? 1 : 0;
  constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
  // nx <= L/2, so the stage-0 inputs x = j + q M with q >= R/2 are always padding
  constexpr int RH = R / 2 > 0 ? R / 2 : 1;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tw0 = tw + L;
  cx<float>* tile = tw0 + L;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  load_twiddles0<L>(tw0, reinterpret_cast<const cx<float>*>(a.tw));
  pdl_wait();  // rho, the gradient, max|G| and the spectra buffer belong to earlier kernels
  const int c = a.comp[blockIdx.y];
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[blockIdx.y] * a.out_cstride;
  const int ntiles = (a.rows + ROWS - 1) / ROWS;
  const float* src = SRC == SRC_VECTOR ? a.vec + c * a.vec_cstride : a.rho;
  const float* m0 = withM0 ? a.M0v + c * a.M0v_cstride : nullptr;
  static_assert(!UPD || (SRC == SRC_RHO_POW && k_per_thread<L>()), "the step is fused into the one-slot pass only");
  // UPD: the gradient rows of the next tile are copied into shared memory (cp.async)
  // while the current tile is separated, at a row stride gs = 8 (mod 16) words so that
  // the two half-warps (rows 2 l and 2 l + 2) read distinct banks
  float* sG = reinterpret_cast<float*>(tile + L * TB);  // [ROWS][gs], nx <= L/2
  const int gs = a.nx + ((8 - a.nx % 16) + 16) % 16;
  float ra[ITER][RH], rb[ITER][RH], ma[ITER][RM ? RH : 1], mb[ITER][RM ? RH : 1];
  bool upd = false;
  float step = 0.0f;
  if constexpr (UPD) {
    upd = true;
    step = a.upd_alpha;
    if (a.upd_normalize) {
      const float gm = __uint_as_float(*a.upd_gmax);
      if (!(gm > 0.0f)) upd = false;  // max|G| = 0: no step
      step = a.upd_alpha / gm;
    }
  }
  auto fetch = [&](int t) {
    const int row0 = t * ROWS;
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      const int j = u % M, line = u / M;
      const int r = row0 + 2 * line;
      const bool ok = NU % kNT == 0 || u < NU;
      const bool va = ok && r < a.rows, vb = ok && r + 1 < a.rows;
      const long long o = (long long)r * a.nx + j;  // x = j of row a; row b follows
      const int xn = a.nx - j;                       // x < nx  <=>  q M < xn
#pragma unroll
      for (int q = 0; q < RH; q++) {
        const bool in_x = q * M < xn;
        ra[it][q] = (in_x && va) ? src[o + q * M] : 0.0f;
        rb[it][q] = (in_x && vb) ? src[o + a.nx + q * M] : 0.0f;
        if constexpr (withM0) {
          ma[it][q] = (in_x && va) ? m0[o + q * M] : 0.0f;
          mb[it][q] = (in_x && vb) ? m0[o + a.nx + q * M] : 0.0f;
        }
      }
    }
    if constexpr (UPD) {
      if (upd) {  // a warp per row: 16-byte pieces when rows start on 16 bytes, else words
        const int nr = min(ROWS, a.rows - row0);
        const float* g = a.upd_G + (long long)row0 * a.nx;
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (a.nx % 4 == 0) {
          for (int rr = w; rr < nr; rr += kNT / 32)
            for (int c = lane; c < a.nx / 4; c += 32) cp16(sG + rr * gs + 4 * c, g + (long long)rr * a.nx + 4 * c);
        } else {
          for (int rr = w; rr < nr; rr += kNT / 32)
            for (int x = lane; x < a.nx; x += 32) cp4(sG + rr * gs + x, g + (long long)rr * a.nx + x);
        }
      }
      cp_commit();
    }
  };
  int t = blockIdx.x;
  if (t < ntiles) fetch(t);
  if constexpr (UPD) cp_wait<0>();
  __syncthreads();
  for (; t < ntiles; t += gridDim.x) {
    const int row0 = t * ROWS;
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (NU % kNT == 0 || u < NU) {
        const int j = u % M, line = u / M;
        cx<float> v[R];
#pragma unroll
        for (int q = RH; q < R; q++) v[q] = zero<float>();
        const int r = row0 + 2 * line;
        const bool wa = r < a.rows, wb = r + 1 < a.rows;
        const long long o = (long long)r * a.nx + j;
        const int xn = a.nx - j;
#pragma unroll
        for (int q = 0; q < RH; q++) {
          float va = ra[it][q], vb = rb[it][q];
          if constexpr (UPD) {
            if (upd && q * M < xn) {
              const float* gl = sG + (2 * line) * gs + j + q * M;
              if (wa) {
                va = fminf(fmaxf(va - step * gl[0], 0.0f), 1.0f);
                a.upd_rho[o + q * M] = va;
              }
              if (wb) {
                vb = fminf(fmaxf(vb - step * gl[gs], 0.0f), 1.0f);
                a.upd_rho[o + a.nx + q * M] = vb;
              }
            }
          }
          if constexpr (SRC != SRC_VECTOR) {
            va = ipow_t<P3>(va, a.p);
            vb = ipow_t<P3>(vb, a.p);
            if constexpr (withM0) {
              va *= ma[it][q];
              vb *= mb[it][q];
            }
          }
          v[q] = mk(va, vb);
        }
        Dft<float, R, false>::run(v);
        twiddle0<L, false>(v, j, tw0);
#pragma unroll
        for (int q = 0; q < R; q++) tile[tix0<M>(j, q, line)] = v[q];
      }
    }
    __syncthreads();
    DifRange<float, L, kNT, 1, S, true>::run(tile, tw);
    if (t + (int)gridDim.x < ntiles) fetch(t + gridDim.x);
    xseparate<L>(tile, out, row0, a.rows, a.P);
    if constexpr (UPD) cp_wait<0>();  // the next tile's gradient rows have landed
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The one-slot pass of rho^p for L = 2 kNT, warp-specialized, with or without a pending
// step (upd_rho set or not): both kinds of evaluation run this one kernel, so the
// spectra of a step-then-evaluate and of the fused step agree bit for bit (separately
// compiled kernels may contract the same products into fused multiply-adds differently).
// One block of 512 threads per SM loops over 32-row tiles. Warps 0-7 take tile r: its
// rho (and gradient) rows arrive by TMA bulk copies (one per row, into rows padded to a
// stride of 8 mod 16 words so that the two half-warps read distinct banks), they apply
// the step if there is one, write the new rho, and run the first DIF stage into one of
// two tiles. Warps 8-15 run
// the second stage of tile r - 1 from the other tile and separate and store its half
// spectra. The stage-0 twiddles of q >= R0/2 are applied by the second group (same
// products); one block barrier per tile.
template <int L>
__host__ __device__ constexpr int xws_pitch(int nx) {
  return nx + ((8 - nx % 16) + 16) % 16;
}
template <int L>
size_t xfwd_ws_smem(int nx) {
  return 128 + (size_t)(2 * L + 2 * L * TB) * sizeof(float2) + (size_t)2 * ROWS * xws_pitch<L>(nx) * sizeof(float) +
         16;
}

template <int L, bool P3>
__global__ void __launch_bounds__(2 * kNT, 1) k_xfwd_ws(XFwdArgs a) {
  using S0 = StageShape<L, 0>;
  using S1 = StageShape<L, 1>;
  static_assert(k_per_thread<L>() && S0::M == TB && S1::R == TB && S1::M == 1, "two-stage plan 32 x 16");
  constexpr int R0 = S0::R, M0 = S0::M, R1 = S1::R, RH = R0 / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tw0 = tw + L;
  cx<float>* tiles = tw0 + L;  // [2][L][TB], swizzled
  const int gp = xws_pitch<L>(a.nx);
  float* srho = reinterpret_cast<float*>(tiles + 2 * L * TB);  // [ROWS][gp]
  float* sg = srho + ROWS * gp;                                  // [ROWS][gp]
  unsigned long long* mb = reinterpret_cast<unsigned long long*>(sg + ROWS * gp);
  for (int i = threadIdx.x; i < L; i += 2 * kNT) tw[i] = reinterpret_cast<const cx<float>*>(a.tw)[i];
  if (threadIdx.x < kNT) load_twiddles0<L>(tw0, reinterpret_cast<const cx<float>*>(a.tw));
  if (threadIdx.x == 0) {
    mbar_init(mb, 1);
    mbar_init_fence();
  }
  pdl_wait();  // rho, the gradient, max|G| and the spectra buffer belong to earlier kernels
  __syncthreads();
  bool upd = a.upd_rho != nullptr;
  float step = a.upd_alpha;
  if (upd && a.upd_normalize) {
    const float gm = __uint_as_float(*a.upd_gmax);
    if (!(gm > 0.0f)) upd = false;  // max|G| = 0: no step
    step = a.upd_alpha / gm;
  }
  const float* rsrc = a.upd_rho ? a.upd_rho : a.rho;
  const int ntiles = (a.rows + ROWS - 1) / ROWS;
  const int nr = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const unsigned rbytes = (unsigned)(a.nx * sizeof(float));
  // thread w < 2 ROWS of group 0: one row copy (rho rows first, then gradient rows); thread 0
  // arms the barrier for all of them first
  auto issue = [&](int r, int t) {
    const int row0 = (blockIdx.x + r * gridDim.x) * ROWS;
    const int n = min(ROWS, a.rows - row0);
    if (t == 0) mbar_expect_tx(mb, (unsigned)(n * (upd ? 2 : 1)) * rbytes);
    bar_named(4, 2 * ROWS);  // the barrier is armed before any copy can complete on it
    if (t < n) bulk_load(srho + t * gp, rsrc + (long long)(row0 + t) * a.nx, rbytes, mb);
    else if (upd && t >= ROWS && t - ROWS < n)
      bulk_load(sg + (t - ROWS) * gp, a.upd_G + (long long)(row0 + t - ROWS) * a.nx, rbytes, mb);
  };
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[0] * a.out_cstride;
  if (threadIdx.x < kNT) {
    // step and first DIF stage of tile r into tiles[r & 1]
    const int t = threadIdx.x;
    const int j = t % M0, line = t / M0;
    if (t < 2 * ROWS) {
      fence_proxy_async_global();  // rho and G were written by earlier kernels with ordinary stores
      if (nr > 0) issue(0, t);
    }
    for (int r = 0; r <= nr; r++) {
      if (r < nr) {
        const int row0 = (blockIdx.x + r * gridDim.x) * ROWS;
        const int rw = row0 + 2 * line;
        const bool wa = rw < a.rows, wb = rw + 1 < a.rows;
        const long long o = (long long)rw * a.nx + j;
        const int xn = a.nx - j;
        mbar_wait(mb, r & 1, a.status);
        float va[RH], vb[RH];
#pragma unroll
        for (int q = 0; q < RH; q++) {
          const bool in_x = q * M0 < xn;
          const float* sr = srho + (2 * line) * gp + j + q * M0;
          const float* sgl = sg + (2 * line) * gp + j + q * M0;
          va[q] = (in_x && wa) ? sr[0] : 0.0f;
          vb[q] = (in_x && wb) ? sr[gp] : 0.0f;
          if (upd) {
            if (in_x && wa) va[q] = fminf(fmaxf(va[q] - step * sgl[0], 0.0f), 1.0f);
            if (in_x && wb) vb[q] = fminf(fmaxf(vb[q] - step * sgl[gp], 0.0f), 1.0f);
          }
        }
        bar_named(2, kNT);  // every thread of the group is done with the staged rows
        if (t < 2 * ROWS && r + 1 < nr) {
          fence_proxy_async_smem();  // those reads before the copies that overwrite them
          issue(r + 1, t);
        }
        cx<float> v[R0];
#pragma unroll
        for (int q = 0; q < RH; q++) {
          if (upd && q * M0 < xn) {
            if (wa) a.upd_rho[o + q * M0] = va[q];
            if (wb) a.upd_rho[o + a.nx + q * M0] = vb[q];
          }
          v[q] = mk(ipow_t<P3>(va[q], a.p), ipow_t<P3>(vb[q], a.p));
        }
        dft32_half_input<false>(v);  // x = j + q M0 >= L/2 is padding
        if (j != 0) {  // q >= R0/2: applied by the other group
#pragma unroll
          for (int q = 1; q < R0 / 2; q++) v[q] = cmul(v[q], tw0[q * M0 + j]);
        }
        cx<float>* tile = tiles + (r & 1) * L * TB;
#pragma unroll
        for (int q = 0; q < R0; q++) tile[tix0<M0>(j, q, line)] = v[q];
      }
      bar_named(1, 2 * kNT);
    }
  } else {
    // second DIF stage of tile r - 1, then its half spectra
    const int t = threadIdx.x - kNT;
    for (int r = 0; r <= nr; r++) {
      if (r >= 1) {
        cx<float>* tile = tiles + ((r - 1) & 1) * L * TB;
#pragma unroll
        for (int it = 0; it < 2; it++) {
          const int u = it * kNT + t, line = u % TB, g = u / TB;
          cx<float> v[R1];
#pragma unroll
          for (int q = 0; q < R1; q++) v[q] = tile[unit_idx<R1, 1, true>(g, g * R1, q, line)];
          if (it == 1) {  // the stage-0 twiddles of g >= R0/2
#pragma unroll
            for (int q = 1; q < R1; q++) v[q] = cmul(v[q], tw[q * g]);
          }
          DftF<R1, false>::run(v);
#pragma unroll
          for (int q = 0; q < R1; q++) tile[unit_idx<R1, 1, true>(g, g * R1, q, line)] = v[q];
        }
        bar_named(3, kNT);  // the tile is transformed
        const int row0 = (blockIdx.x + (r - 1) * gridDim.x) * ROWS;
        const int k = t, nrow = a.rows - row0;
        const int pa = pos_of_k<L>(k), pb = pos_of_k<L>((L - k) % L);
        const cx<float>* ta = tile + pa * TB;
        const cx<float>* tb = tile + pb * TB;
        const int ca = swz(pa), cb = swz(pb);
        cx<float>* dst = out + (long long)row0 * a.P + k;
#pragma unroll
        for (int l = 0; l < TB; l++) {
          const cx<float> Z = ta[l ^ ca], Zm = tb[l ^ cb];
          if (2 * l < nrow) dst[(2 * l) * a.P] = mk(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
          if (2 * l + 1 < nrow) dst[(2 * l + 1) * a.P] = mk(0.5f * (Z.y + Zm.y), 0.5f * (Zm.x - Z.x));
        }
        const int W = a.P - L / 2, pn = pos_of_k<L>(L / 2);
        for (int rr = t / 16; rr < 2 * TB && rr < nrow; rr += kNT / 16) {
          for (int c = t % 16; c < W; c += 16) {
            cx<float> v = zero<float>();
            if (c == 0) {
              const cx<float> Z = tile[tix(pn, rr >> 1)];
              v = (rr & 1) ? mk(Z.y, 0.0f) : mk(Z.x, 0.0f);
            }
            out[(long long)(row0 + rr) * a.P + L / 2 + c] = v;
          }
        }
      }
      bar_named(1, 2 * kNT);
    }
  }
}

template <int L, bool P3>
int run_xfwd_ws(const XFwdArgs& a, cudaStream_t s) {
  const size_t sm = xfwd_ws_smem<L>(a.nx);
  static size_t init = 0;
  if (init < sm) {
    if (cudaFuncSetAttribute(k_xfwd_ws<L, P3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = sm;
  }
  const int ntiles = (a.rows + ROWS - 1) / ROWS;
  if (ntiles <= 0) return 0;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  const int blocks = ntiles < nsm ? ntiles : nsm;
  return launch_k(k_xfwd_ws<L, P3>, dim3(blocks), dim3(2 * kNT), sm, s, a.pdl != 0, a) == cudaSuccess ? 0 : -1;
}

template <int L, int SRC, bool P3, bool UPD = false>
int run_xfwd_src(const XFwdArgs& a, int ncomp, cudaStream_t s) {
  const size_t sm = xsmem<L>() + (UPD ? (size_t)ROWS * (L / 2 + 15) * sizeof(float) : 0);
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xfwd<L, SRC, P3, UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  const int tiles = (a.rows + ROWS - 1) / ROWS;
  if (tiles == 0 || ncomp == 0) return 0;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 148;
  }
  const int per_comp = (2 * nsm + ncomp - 1) / ncomp;  // two resident blocks per SM in total
  const int blocks = tiles < per_comp ? tiles : per_comp;
  return launch_k(k_xfwd<L, SRC, P3, UPD>, dim3(blocks, ncomp), dim3(kNT), sm, s, a.pdl != 0, a) == cudaSuccess ? 0
                                                                                                       : -1;
}
template <int L, int SRC>
int run_xfwd_pow(const XFwdArgs& a, int ncomp, cudaStream_t s) {
  if constexpr (k_per_thread<L>()) {
    if constexpr (SRC == SRC_RHO_POW) {
      if (a.upd_rho && ncomp != 1) return -1;
      // warp-specialized form, with or without the step: rows start on 16 bytes (row
      // copies) and fit the staging
      if (ncomp == 1 && a.nx % 4 == 0 && xfwd_ws_smem<L>(a.nx) <= 227 * 1024 &&
          ((reinterpret_cast<uintptr_t>(a.upd_rho ? a.upd_rho : a.rho) | reinterpret_cast<uintptr_t>(a.upd_G)) &
           15) == 0)
        return a.p == 3.0f ? run_xfwd_ws<L, true>(a, s) : run_xfwd_ws<L, false>(a, s);
      if (a.upd_rho)
        return a.p == 3.0f ? run_xfwd_src<L, SRC, true, true>(a, ncomp, s)
                           : run_xfwd_src<L, SRC, false, true>(a, ncomp, s);
    }
    if (a.p == 3.0f) return run_xfwd_src<L, SRC, true>(a, ncomp, s);
  }
  if (a.upd_rho) return -1;  // no fused step for this length or source
  return run_xfwd_src<L, SRC, false>(a, ncomp, s);
}
template <int L>
int run_xfwd(const XFwdArgs& a, int ncomp, cudaStream_t s) {
  if (a.src == SRC_RHO_POW) return run_xfwd_pow<L, SRC_RHO_POW>(a, ncomp, s);
  if (a.src == SRC_RHO_M0) return run_xfwd_pow<L, SRC_RHO_M0>(a, ncomp, s);
  if (a.upd_rho) return -1;
  return run_xfwd_src<L, SRC_VECTOR, false>(a, ncomp, s);
}

}  // namespace

bool xfwd_fuses_step(int L, int src, int ncomp) { return L == 2 * kNT && src == SRC_RHO_POW && ncomp == 1; }

int launch_xfwd(int L, const XFwdArgs& a, int ncomp, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_xfwd<LL>(a, ncomp, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

}  // namespace tmk
