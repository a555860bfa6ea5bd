// Inverse x pass of the stray-field convolution (Sec. "Discretization", Eq. (convolution)).
//
// Half spectra are extended by Hermitian symmetry, two rows are recovered from one
// complex inverse transform, cropped to nx, and handed to a sink: write H; the
// least-squares objective and dJ/dH, whose zero-padded forward x transform (the
// adjoint source) starts in the same registers; or the chain rule
// dJ/drho = p rho^(p-1) M0 . (D g) (Sec. "Methodology", Eqs. (adjoint1)-(adjoint2)).
// The last inverse stage maps consecutive threads to consecutive x of one row pair,
// so global rows are written in 64-byte runs straight from registers.
#include "tma.cuh"
#include "xpass.cuh"

namespace tmk {

namespace {

// Called by every thread of every block after thread 0 wrote the block's J partial:
// the last block to finish sums the partials in index order (the order of a separate
// one-block reduction) into *Jout and re-arms the counter.
__device__ void finish_j(const XInvArgs& a) {
  __shared__ unsigned int last;
  __shared__ double r2[kNT];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(a.Jcount, 1u) == gridDim.x * gridDim.y - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int n = gridDim.x * gridDim.y;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kNT) s += __ldcg(a.Jpart + i);
  r2[threadIdx.x] = s;
  __syncthreads();
  for (int w = kNT / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) r2[threadIdx.x] += r2[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *a.Jout = r2[0];
    *a.Jcount = 0u;
  }
}

// P3: p = 3 fixed at compile time (chain sink with one contracted slot only). ONE: the
// chain sink of one slot already contracted with the constant M0; else every slot with
// its M0 component (MINB: the blocks per SM the registers are sized for).
template <int L, int SINK, int MINB, bool P3, bool ONE>
__global__ void __launch_bounds__(kNT, MINB) k_xinv(XInvArgs a) {
  constexpr int S = plan_stages(L);
  using S0 = StageShape<L, 0>;
  constexpr int R = S0::R, M = S0::M, NU = M * TB, ITER = (NU + kNT - 1) / kNT;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tw0 = tw + L;
  cx<float>* tile = tw0 + L;
  __shared__ double red[kNT / 32];
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  load_twiddles0<L>(tw0, reinterpret_cast<const cx<float>*>(a.tw));
  pdl_wait();  // the spectra, rho and the outputs belong to earlier kernels
  const int row0 = a.row_base + blockIdx.x * ROWS;
  const cx<float>* in0 = reinterpret_cast<const cx<float>*>(a.in);

  if constexpr (SINK == SINK_CHAIN && ONE) {
    // one slot, already contracted with the constant M0: G = p rho^(p-1) D
    constexpr int RH = R / 2 > 0 ? R / 2 : 1;  // x = j + q M < nx <= L/2 needs q < R/2
    __shared__ float wmax[kNT / 32];
    __syncthreads();
    xhermitian<L>(tile, in0 + a.in_slot[0] * a.in_cstride, row0, a.rows, a.P);
    // p rho^(p-1) of this tile, fetched while the inverse stages run
    float pa[ITER][RH], pb[ITER][RH];
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      const int j = u % M, line = u / M;
      const int r = row0 + 2 * line;
      const bool ok = NU % kNT == 0 || u < NU;
      const bool va = ok && r < a.rows, vb = ok && r + 1 < a.rows;
      const long long o = (long long)r * a.nx + j;
      const int xn = a.nx - j;
#pragma unroll
      for (int q = 0; q < RH; q++) {
        const bool in_x = q * M < xn;
        pa[it][q] = (in_x && va) ? a.rho[o + q * M] : 0.0f;
        pb[it][q] = (in_x && vb) ? a.rho[o + a.nx + q * M] : 0.0f;
      }
    }
    __syncthreads();
    DitRange<float, L, kNT, 1, S, true>::run(tile, tw);
    float gm = 0.0f;
    xdit0<L>(tile, tw0, [&](int it, int j, int line, cx<float>* v) {
      const int r = row0 + 2 * line;
      const bool va = r < a.rows, vb = r + 1 < a.rows;
      float* g = a.G + (long long)r * a.nx + j;
      const int xn = a.nx - j;
#pragma unroll
      for (int q = 0; q < RH; q++) {
        if (q * M >= xn) continue;
        if (va) {
          const float G = dpow_t<P3>(pa[it][q], a.p) * v[q].x;
          g[q * M] = G;
          gm = fmaxf(gm, fabsf(G));
        }
        if (vb) {
          const float G = dpow_t<P3>(pb[it][q], a.p) * v[q].y;
          g[a.nx + q * M] = G;
          gm = fmaxf(gm, fabsf(G));
        }
      }
      return false;
    });
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kNT / 32; w++) gm = fmaxf(gm, wmax[w]);
      if (gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    }
    return;
  } else if constexpr (SINK == SINK_CHAIN && R == 2 * TB && M == TB && ITER == 1) {
    // every slot with its M0 component, L = 512 = 32 x 16: the last inverse stage forms only
    // the outputs x = j + q M < L/2 (q < R/2; nx <= L/2), and the sums over the slots stay in
    // registers for those
    constexpr int RH = R / 2;
    const int j = threadIdx.x % M, line = threadIdx.x / M;
    const int ra = row0 + 2 * line, rb = ra + 1;
    float acc[RH][2];
#pragma unroll
    for (int q = 0; q < RH; q++) acc[q][0] = acc[q][1] = 0.0f;
    for (int jc = 0; jc < a.ncomp; jc++) {
      __syncthreads();
      xhermitian<L>(tile, in0 + a.in_slot[jc] * a.in_cstride, row0, a.rows, a.P);
      __syncthreads();
      DitRange<float, L, kNT, 1, S, true>::run(tile, tw);
      const int c = a.comp[jc];
      cx<float> v[R];
#pragma unroll
      for (int q = 0; q < R; q++) v[q] = tile[tix0<M>(j, q, line)];
      twiddle0<L, true>(v, j, tw0);
      dft_low_half<R, true>(v);
#pragma unroll
      for (int q = 0; q < RH; q++) {
        const int x = j + q * M;
        float ma = 1.0f, mb = 1.0f;  // contracted slot: coefficient 1
        if (a.M0v && x < a.nx) {
          if (ra < a.rows) ma = a.M0v[c * a.M0v_cstride + (long long)ra * a.nx + x];
          if (rb < a.rows) mb = a.M0v[c * a.M0v_cstride + (long long)rb * a.nx + x];
        }
        acc[q][0] += ma * v[q].x;
        acc[q][1] += mb * v[q].y;
      }
    }
    float gm = 0.0f;
#pragma unroll
    for (int q = 0; q < RH; q++) {
      const int x = j + q * M;
      if (x >= a.nx) continue;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int row = ra + h;
        if (row >= a.rows) continue;
        const long long o = (long long)row * a.nx + x;
        const float G = dpow(a.rho[o], a.p) * acc[q][h];
        a.G[o] = G;
        gm = fmaxf(gm, fabsf(G));
      }
    }
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((threadIdx.x & 31) == 0 && gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    return;
  } else if constexpr (SINK == SINK_CHAIN) {
    float acc[ITER][R][2];
#pragma unroll
    for (int it = 0; it < ITER; it++)
#pragma unroll
      for (int q = 0; q < R; q++) acc[it][q][0] = acc[it][q][1] = 0.0f;
    for (int jc = 0; jc < a.ncomp; jc++) {
      __syncthreads();
      xhermitian<L>(tile, in0 + a.in_slot[jc] * a.in_cstride, row0, a.rows, a.P);
      __syncthreads();
      DitRange<float, L, kNT, 1, S, true>::run(tile, tw);
      const int c = a.comp[jc];
      xdit0<L>(tile, tw0, [&](int it, int j, int line, cx<float>* v) {
        const int ra = row0 + 2 * line, rb = ra + 1;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int x = j + q * M;
          float ma = 1.0f, mb = 1.0f;  // contracted slot: coefficient 1
          if (a.M0v && x < a.nx) {
            if (ra < a.rows) ma = a.M0v[c * a.M0v_cstride + (long long)ra * a.nx + x];
            if (rb < a.rows) mb = a.M0v[c * a.M0v_cstride + (long long)rb * a.nx + x];
          }
          acc[it][q][0] += ma * v[q].x;
          acc[it][q][1] += mb * v[q].y;
        }
        return false;
      });
    }
    float gm = 0.0f;
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (NU % kNT == 0 || u < NU) {
        const int j = u % M, line = u / M;
        const int ra = row0 + 2 * line;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int x = j + q * M;
          if (x >= a.nx) continue;
#pragma unroll
          for (int h = 0; h < 2; h++) {
            const int row = ra + h;
            if (row >= a.rows) continue;
            const long long o = (long long)row * a.nx + x;
            const float G = dpow(a.rho[o], a.p) * acc[it][q][h];
            a.G[o] = G;
            gm = fmaxf(gm, fabsf(G));
          }
        }
      }
    }
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((threadIdx.x & 31) == 0 && gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    return;
  } else {
    const int jc = blockIdx.y, c = a.comp[jc];
    const cx<float>* in = in0 + a.in_slot[jc] * a.in_cstride;
    if constexpr (SINK == SINK_OBJECTIVE) {
      if (a.ext) {  // only the rows of the target planes carry H (and the adjoint source)
        const long long lo = (long long)a.ext[0] * a.ny, hi = (long long)a.ext[1] * a.ny;
        if (row0 + ROWS <= lo || row0 >= hi) {
          if (threadIdx.x == 0) a.Jpart[jc * gridDim.x + blockIdx.x] = 0.0;
          if (a.Jcount) finish_j(a);
          return;
        }
      }
    }
    __syncthreads();
    xhermitian<L>(tile, in, row0, a.rows, a.P);
    __syncthreads();
    DitRange<float, L, kNT, 1, S, true>::run(tile, tw);

    if constexpr (SINK == SINK_FIELD) {
      xdit0<L>(tile, tw0, [&](int, int j, int line, cx<float>* v) {
        const int ra = row0 + 2 * line, rb = ra + 1;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int x = j + q * M;
          if (x >= a.nx) continue;
          if (ra < a.rows) a.H[c * a.H_cstride + (long long)ra * a.nx + x] = v[q].x;
          if (rb < a.rows) a.H[c * a.H_cstride + (long long)rb * a.nx + x] = v[q].y;
        }
        return false;
      });
      return;
    } else {
      // SINK_OBJECTIVE: J partial; g_c = 2 w_c (H_c - Ht_c) on the mask, zero elsewhere and
      // for x >= nx (the padding); the forward stage 0 of the adjoint source runs on g
      const float wc = a.w[c];
      double jacc = 0.0;
      int mine = 0;
      xdit0<L>(tile, tw0, [&](int, int j, int line, cx<float>* v) {
        const int ra = row0 + 2 * line;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int x = j + q * M;
          float g[2] = {0.0f, 0.0f};
          if (x < a.nx) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
              const int row = ra + h;
              if (row >= a.rows) continue;
              const long long o = (long long)row * a.nx + x;
              const float hv = h ? v[q].y : v[q].x;
              if (a.H) a.H[c * a.H_cstride + o] = hv;
              if (wc != 0.0f && a.mask[o]) {
                mine = 1;
                const float r = hv - (a.Ht ? a.Ht[c * a.Ht_cstride + o] : a.Htc[c]);
                jacc += (double)wc * (double)r * (double)r;
                g[h] = 2.0f * wc * r;
              }
            }
          }
          v[q] = mk(g[0], g[1]);
        }
        return true;
      });
      for (int off = 16; off > 0; off >>= 1) jacc += __shfl_xor_sync(0xffffffffu, jacc, off);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = jacc;
      const int any_mask = __syncthreads_or(mine);
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNT / 32; w++) s += red[w];
        a.Jpart[jc * gridDim.x + blockIdx.x] = s;
      }
      if (a.Jcount) finish_j(a);
      if (!a.adj_out) return;
      cx<float>* adj = reinterpret_cast<cx<float>*>(a.adj_out) + a.in_slot[jc] * a.in_cstride;
      if (!any_mask) {  // the adjoint source vanishes on all rows of this block
        for (int i = threadIdx.x; i < ROWS * a.P; i += kNT) {
          const int rr = i / a.P, k = i - rr * a.P, row = row0 + rr;
          if (row < a.rows) adj[(long long)row * a.P + k] = zero<float>();
        }
        return;
      }
      DifRange<float, L, kNT, 1, S, true>::run(tile, tw);
      xseparate<L>(tile, adj, row0, a.rows, a.P);
    }
  }
}

// ---------------------------------------------------------------------------
// Chain rule for L = 2 kNT with one contracted slot, warp-specialized: a block of 512
// threads per SM loops over 32-row tiles; warps 0-7 build the Hermitian extension of
// tile r from its spectrum rows (one TMA bulk copy into shared memory, a tile ahead)
// and run the first inverse stage into one of two tiles, while warps 8-15 run the last
// inverse stage of tile r - 1 from the other and apply G = p rho^(p-1) D, with rho
// loaded into registers a round ahead. The stage-0 twiddles are shared as in the fused
// y/z kernels (same products, same results). One block barrier per tile.
template <int L>
constexpr size_t xinv_ws_smem(int P) {
  return 128 + (size_t)(2 * L + 2 * L * TB) * sizeof(float2) + (size_t)ROWS * P * sizeof(float2) + 16;
}

template <int L, bool P3>
__global__ void __launch_bounds__(2 * kNT, 1) k_xinv_ws(XInvArgs a) {
  using S0 = StageShape<L, 0>;
  using S1 = StageShape<L, 1>;
  static_assert(k_per_thread<L>() && S0::M == TB && S1::R == TB && S1::M == 1, "two-stage plan 32 x 16");
  constexpr int R0 = S0::R, M0 = S0::M, R1 = S1::R, RH = R0 / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tw0 = tw + L;
  cx<float>* tiles = tw0 + L;                       // [2][L][TB], swizzled
  cx<float>* raw = tiles + 2 * L * TB;              // [ROWS][P] spectrum rows of the next tile
  unsigned long long* mb = reinterpret_cast<unsigned long long*>(raw + ROWS * a.P);
  __shared__ float wmax[kNT / 32];
  for (int i = threadIdx.x; i < L; i += 2 * kNT) tw[i] = reinterpret_cast<const cx<float>*>(a.tw)[i];
  if (threadIdx.x < kNT) load_twiddles0<L>(tw0, reinterpret_cast<const cx<float>*>(a.tw));
  if (threadIdx.x == 0) {
    mbar_init(mb, 1);
    mbar_init_fence();
  }
  pdl_wait();  // the spectra, rho and G belong to earlier kernels
  __syncthreads();
  const int ntiles = (a.rows + ROWS - 1) / ROWS;
  const int nr = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.in) + a.in_slot[0] * a.in_cstride;
  auto issue = [&](int r) {  // spectrum rows of tile blockIdx.x + r gridDim.x, one bulk copy
    const int row0 = (blockIdx.x + r * gridDim.x) * ROWS;
    const int n = min(ROWS, a.rows - row0);
    mbar_expect_tx(mb, (unsigned)(n * a.P * sizeof(float2)));
    bulk_load(raw, in + (long long)row0 * a.P, (unsigned)(n * a.P * sizeof(float2)), mb);
  };
  if (threadIdx.x < kNT) {
    // Hermitian extension and first inverse stage of tile r into tiles[r & 1]
    const int t = threadIdx.x;
    // the spectrum rows were written by the previous kernel through ordinary stores; make
    // them visible to the tensor-copy (async) proxy before its first read
    if (t == 0) asm volatile("fence.proxy.async.global;\n" ::: "memory");
    if (t == 0 && nr > 0) issue(0);
    const int k = t;  // one frequency per thread
    const int pa = pos_of_k<L>(k), pb = pos_of_k<L>((L - k) % L), pn = pos_of_k<L>(L / 2);
    const int ca = swz(pa), cb = swz(pb);
    for (int r = 0; r <= nr; r++) {
      if (r < nr) {
        const int row0 = (blockIdx.x + r * gridDim.x) * ROWS;
        const int nrow = a.rows - row0;
        cx<float>* tile = tiles + (r & 1) * L * TB;
        mbar_wait(mb, r & 1, a.status);
        cx<float> A[TB], B[TB];
#pragma unroll
        for (int l = 0; l < TB; l++) {
          A[l] = 2 * l < nrow ? raw[(2 * l) * a.P + k] : zero<float>();
          B[l] = 2 * l + 1 < nrow ? raw[(2 * l + 1) * a.P + k] : zero<float>();
        }
        cx<float> An = zero<float>(), Bn = zero<float>();  // k = L/2 of line t
        if (t < TB) {
          if (2 * t < nrow) An = raw[(2 * t) * a.P + L / 2];
          if (2 * t + 1 < nrow) Bn = raw[(2 * t + 1) * a.P + L / 2];
        }
        bar_named(2, kNT);  // every thread of the group is done with the raw rows
        if (t == 0 && r + 1 < nr) {
          fence_proxy_async_smem();  // those reads before the copy that overwrites them
          issue(r + 1);
        }
        cx<float>* ta = tile + pa * TB;
        cx<float>* tb = tile + pb * TB;
        if (k == 0) {
#pragma unroll
          for (int l = 0; l < TB; l++) ta[l ^ ca] = mk(A[l].x, B[l].x);
        } else {
#pragma unroll
          for (int l = 0; l < TB; l++) {
            ta[l ^ ca] = mk(A[l].x - B[l].y, A[l].y + B[l].x);  // A + iB
            tb[l ^ cb] = mk(A[l].x + B[l].y, B[l].x - A[l].y);  // conj(A) + i conj(B)
          }
        }
        if (t < TB) tile[tix(pn, t)] = mk(An.x, Bn.x);
        bar_named(2, kNT);  // the tile is complete
        // first inverse stage (positions g R1 + q, 2 kNT units); the stage-0 twiddles of
        // g >= R0/2 are applied here
#pragma unroll
        for (int it = 0; it < 2; it++) {
          const int u = it * kNT + t, line = u % TB, g = u / TB;
          cx<float> v[R1];
#pragma unroll
          for (int q = 0; q < R1; q++) v[q] = tile[unit_idx<R1, 1, true>(g, g * R1, q, line)];
          DftF<R1, true>::run(v);
          if (it == 1) {
#pragma unroll
            for (int q = 1; q < R1; q++) v[q] = cmulc(v[q], tw[q * g]);
          }
#pragma unroll
          for (int q = 0; q < R1; q++) tile[unit_idx<R1, 1, true>(g, g * R1, q, line)] = v[q];
        }
      }
      bar_named(1, 2 * kNT);
    }
  } else {
    // last inverse stage of tile r - 1 and the chain rule
    const int t = threadIdx.x - kNT;
    const int j = t % M0, line = t / M0;
    float pa[RH], pb[RH];
    auto fetch_rho = [&](int r) {
      const int rw = (blockIdx.x + r * gridDim.x) * ROWS + 2 * line;
      const bool va = rw < a.rows, vb = rw + 1 < a.rows;
      const long long o = (long long)rw * a.nx + j;
      const int xn = a.nx - j;
#pragma unroll
      for (int q = 0; q < RH; q++) {
        const bool in_x = q * M0 < xn;
        pa[q] = (in_x && va) ? a.rho[o + q * M0] : 0.0f;
        pb[q] = (in_x && vb) ? a.rho[o + a.nx + q * M0] : 0.0f;
      }
    };
    if (nr > 0) fetch_rho(0);
    float gm = 0.0f;
    for (int r = 0; r <= nr; r++) {
      if (r >= 1) {
        const cx<float>* tile = tiles + ((r - 1) & 1) * L * TB;
        cx<float> v[R0];
#pragma unroll
        for (int q = 0; q < R0; q++) v[q] = tile[tix0<M0>(j, q, line)];
        if (j != 0) {  // q >= R0/2: applied by the other group
#pragma unroll
          for (int q = 1; q < R0 / 2; q++) v[q] = cmulc(v[q], tw0[q * M0 + j]);
        }
        dft_low_half<R0, true>(v);  // x = j + q M0 < L/2: the first half of the outputs
        const int rw = (blockIdx.x + (r - 1) * gridDim.x) * ROWS + 2 * line;
        const bool va = rw < a.rows, vb = rw + 1 < a.rows;
        float* g = a.G + (long long)rw * a.nx + j;
        const int xn = a.nx - j;
#pragma unroll
        for (int q = 0; q < RH; q++) {
          if (q * M0 >= xn) continue;
          if (va) {
            const float G = dpow_t<P3>(pa[q], a.p) * v[q].x;
            g[q * M0] = G;
            gm = fmaxf(gm, fabsf(G));
          }
          if (vb) {
            const float G = dpow_t<P3>(pb[q], a.p) * v[q].y;
            g[a.nx + q * M0] = G;
            gm = fmaxf(gm, fabsf(G));
          }
        }
        if (r < nr) fetch_rho(r);  // rho of the tile the other group is preparing
      }
      bar_named(1, 2 * kNT);
    }
    for (int off = 16; off > 0; off >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if ((t & 31) == 0) wmax[t >> 5] = gm;
    bar_named(3, kNT);
    if (t == 0) {
      for (int w = 1; w < kNT / 32; w++) gm = fmaxf(gm, wmax[w]);
      if (gm > 0.0f) atomicMax(a.gmax, __float_as_uint(gm));
    }
  }
}

template <int L, bool P3>
int run_xinv_ws(const XInvArgs& a, cudaStream_t s) {
  const size_t sm = xinv_ws_smem<L>(a.P);
  static size_t init = 0;
  if (init < sm) {
    if (cudaFuncSetAttribute(k_xinv_ws<L, P3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
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
  return launch_k(k_xinv_ws<L, P3>, dim3(blocks), dim3(2 * kNT), sm, s, a.pdl != 0, a) == cudaSuccess ? 0 : -1;
}

template <int L, int SINK, int MINB, bool P3, bool ONE = false>
int run_xinv_sink(const XInvArgs& a, cudaStream_t s) {
  const size_t sm = xsmem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_xinv<L, SINK, MINB, P3, ONE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -1;
    init = true;
  }
  const int blocks = (a.rows - a.row_base + ROWS - 1) / ROWS;
  if (blocks <= 0 || a.ncomp == 0) return 0;
  const int gy = SINK == SINK_CHAIN ? 1 : a.ncomp;
  return launch_k(k_xinv<L, SINK, MINB, P3, ONE>, dim3(blocks, gy), dim3(kNT), sm, s, a.pdl != 0, a) == cudaSuccess ? 0
                                                                                                        : -1;
}
template <int L>
int run_xinv(const XInvArgs& a, cudaStream_t s) {
  if (a.sink == SINK_FIELD) return run_xinv_sink<L, SINK_FIELD, 2, false>(a, s);
  if (a.sink == SINK_OBJECTIVE) return run_xinv_sink<L, SINK_OBJECTIVE, 2, false>(a, s);
  if (a.ncomp == 1 && a.M0v == nullptr) {  // contracted slot
    if constexpr (k_per_thread<L>()) {
      // warp-specialized form when the block's raw rows fit beside the two tiles
      if (a.row_base == 0 && xinv_ws_smem<L>(a.P) <= 227 * 1024 && (reinterpret_cast<uintptr_t>(a.in) & 15) == 0)
        return a.p == 3.0f ? run_xinv_ws<L, true>(a, s) : run_xinv_ws<L, false>(a, s);
      if (a.p == 3.0f) return run_xinv_sink<L, SINK_CHAIN, 2, true, true>(a, s);
    }
    return run_xinv_sink<L, SINK_CHAIN, 2, false, true>(a, s);
  }
  // every slot with its M0 component; L = 512: three blocks per SM (at 256^3 with a varying
  // M0 the pass took 665 us forming all 32 outputs per unit with one block per SM, 327 us
  // with the low half and two, 304 us with three, despite the spills)
  if constexpr (StageShape<L, 0>::R == 2 * TB && StageShape<L, 0>::M == TB)
    return run_xinv_sink<L, SINK_CHAIN, 3, false, false>(a, s);
  return run_xinv_sink<L, SINK_CHAIN, 1, false, false>(a, s);
}

}  // namespace

int xinv_rows_per_block() { return ROWS; }

int launch_xinv(int L, const XInvArgs& a, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_xinv<LL>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

}  // namespace tmk
