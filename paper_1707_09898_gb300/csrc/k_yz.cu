// y and z passes of the stray-field convolution (Sec. "Discretization", Eq. (convolution)).
//
// y pass: tiles of 16 contiguous kx columns of one component; forward
// transforms read y < n_in (the rest of the length-L line is the zero padding)
// and write all L digit-reversed positions; inverse transforms read all
// positions and keep the first n_out rows (the crop).
// z pass: forward z transform, the product with the tensor N^(k) (real, stored
// once for kx, ky, kz in [0, L/2] and unfolded by parity), inverse z transform,
// fused per column so the spectra never leave shared memory. The product is
// written as out_o = sum_i s_oi in_i with s_oi = v_o^T N^ u_i: u_i, v_o are unit
// vectors for plain components, or M0 when the magnetization (forward input) or
// the chain rule (adjoint output) is contracted with a constant M0 -- exact by
// linearity of the convolution, and it removes two of the three transforms.
// One input: one block per (column tile, output). Several inputs: a cluster of
// one block per input; the blocks exchange spectra through distributed shared
// memory.
#include <cooperative_groups.h>

#include "fft.cuh"
#include "internal.h"
#include "unet_tc.cuh"

namespace cg = cooperative_groups;

namespace tmk {

namespace {

// Two-stage plans with R0 = 2 R1 = 2 M0 = 32 (L = 512 = 32 x 16): the radix-32 stage of an
// input whose upper half is zero runs as two 16-point DFTs (dft32_half_input), and an
// inverse whose upper half is cropped forms only its lower half (dft_low_half).
template <int L>
__host__ __device__ constexpr bool zmulti_plan() {
  return plan_stages(L) == 2 && StageShape<L, 0>::R == 2 * StageShape<L, 1>::R &&
         StageShape<L, 0>::M == StageShape<L, 1>::R && StageShape<L, 1>::R == TB;
}

template <int L, bool INV>
__global__ void __launch_bounds__(kNT, 3) k_ypass(YArgs a) {
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  pdl_wait();  // the input planes, the plane extent and the outputs belong to earlier kernels
  const int chunk = blockIdx.x;
  int z = a.z0 + blockIdx.y;
  if (a.ext) {
    z += a.ext[0];
    if (z >= a.ext[1]) return;
  }
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.in) + a.in_slot[blockIdx.z] * a.in_cstride +
                        z * a.in_zstride + chunk * TB;
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[blockIdx.z] * a.out_cstride +
                   z * a.out_zstride + chunk * TB;
  __syncthreads();
  if constexpr (zmulti_plan<L>()) {
    using S1 = StageShape<L, 1>;
    constexpr int R0 = StageShape<L, 0>::R, M0 = StageShape<L, 0>::M, R1 = S1::R;
    const int line = threadIdx.x % TB, j = threadIdx.x / TB;
    if (!INV && a.n_in <= L / 2) {
      {  // stage 0: rows y = j + q M0 < n_in (<= L/2) in
        cx<float> v[R0];
#pragma unroll
        for (int q = 0; q < R0 / 2; q++) {
          const int y = j + q * M0;
          v[q] = y < a.n_in ? in[y * a.in_pstride + line] : zero<float>();
        }
        dft32_half_input<false>(v);
        if (j != 0) {
#pragma unroll
          for (int q = 1; q < R0; q++) v[q] = cmul(v[q], tw[j * q]);
        }
#pragma unroll
        for (int q = 0; q < R0; q++) tile[(j + q * M0) * TB + line] = v[q];
      }
      __syncthreads();
#pragma unroll
      for (int it = 0; it < 2; it++) {  // last stage: units g, positions g R1 + q out
        const int g = it * (R0 / 2) + j;
        cx<float> v[R1];
#pragma unroll
        for (int q = 0; q < R1; q++) v[q] = tile[(g * R1 + q) * TB + line];
        DftF<R1, false>::run(v);
#pragma unroll
        for (int q = 0; q < R1; q++) out[(g * R1 + q) * a.out_pstride + line] = v[q];
      }
      return;
    }
    if (INV && a.n_out <= L / 2) {
#pragma unroll
      for (int it = 0; it < 2; it++) {  // first inverse stage: units g, positions g R1 + q in
        const int g = it * (R0 / 2) + j;
        cx<float> v[R1];
#pragma unroll
        for (int q = 0; q < R1; q++) v[q] = in[(g * R1 + q) * a.in_pstride + line];
        DftF<R1, true>::run(v);
#pragma unroll
        for (int q = 0; q < R1; q++) tile[(g * R1 + q) * TB + line] = v[q];
      }
      __syncthreads();
      cx<float> v[R0];  // last inverse stage: rows y = j + q M0 < n_out (<= L/2) out
#pragma unroll
      for (int q = 0; q < R0; q++) v[q] = tile[(j + q * M0) * TB + line];
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R0; q++) v[q] = cmulc(v[q], tw[j * q]);
      }
      dft_low_half<R0, true>(v);
#pragma unroll
      for (int q = 0; q < R0 / 2; q++) {
        const int y = j + q * M0;
        if (y < a.n_out) out[y * a.out_pstride + line] = v[q];
      }
      return;
    }
  }
  if (!INV) {
    dif_stage0_load<float, L, kNT>(tile, tw, [&](int pos, int line) {
      return pos < a.n_in ? in[pos * a.in_pstride + line] : zero<float>();
    });
    __syncthreads();
    DifRange<float, L, kNT, 1, S - 1>::run(tile, tw);
    dif_last_store<float, L, kNT>(tile, [&](int pos, int line, cx<float> v) { out[pos * a.out_pstride + line] = v; });
  } else {
    dit_last_load<float, L, kNT>(tile, [&](int pos, int line) { return in[pos * a.in_pstride + line]; });
    __syncthreads();
    DitRange<float, L, kNT, 1, S - 1>::run(tile, tw);
    dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
      if (pos < a.n_out) out[pos * a.out_pstride + line] = v;
    });
  }
}

// Tensor factor s(k) = sum_c coef[c] N^_c(k) for the column (ky, kx): the folded
// storage holds kx, ky, kz in [0, L/2]; odd components change sign under
// ky -> Ly - ky and kz -> Lz - kz (kx <= Lx/2 always).
struct TensorCol {
  const float* T;  // T + kyf * P + kx
  long long Tc, Tz;
  float sy;
  int need, single;  // bitmask of components; index if exactly one is needed, else -1
  float coef[6];
  float c1;          // coef[single] (no run-time index into coef)
  __device__ __forceinline__ float at(int kz, int Lz) const {
    const bool lo = kz <= Lz / 2;
    const int kzf = lo ? kz : Lz - kz;
    const float sz = lo ? 1.0f : -1.0f;
    const float* t = T + kzf * Tz;
    if (single >= 0) {
      const float sg = single == 3 ? sy : single == 4 ? sz : single == 5 ? sy * sz : 1.0f;
      return c1 * sg * t[single * Tc];
    }
    float r = 0.0f;
    if (need & 1) r += coef[0] * t[0];
    if (need & 2) r += coef[1] * t[Tc];
    if (need & 4) r += coef[2] * t[2 * Tc];
    if (need & 8) r += coef[3] * sy * t[3 * Tc];
    if (need & 16) r += coef[4] * sz * t[4 * Tc];
    if (need & 32) r += coef[5] * sy * sz * t[5 * Tc];
    return r;
  }
};

__device__ __forceinline__ TensorCol make_tcol(const ZArgs& a, int o, int i, int kyf, float sy, long long kx0) {
  TensorCol t;
  t.T = a.T + kyf * (long long)a.P + kx0;
  t.Tc = a.Tc;
  t.Tz = a.Tz;
  t.sy = sy;
  t.need = 0;
#pragma unroll
  for (int c = 0; c < 6; c++) {  // (o, i) selected by compile-time indexes: no local copy of a.coef
    float v = 0.0f;
#pragma unroll
    for (int oo = 0; oo < 3; oo++)
#pragma unroll
      for (int ii = 0; ii < 3; ii++)
        if (oo == o && ii == i) v = a.coef[oo][ii][c];
    t.coef[c] = v;
    if (v != 0.0f) t.need |= 1 << c;
  }
  t.single = (t.need != 0 && (t.need & (t.need - 1)) == 0) ? __ffs(t.need) - 1 : -1;
  t.c1 = 0.0f;
#pragma unroll
  for (int c = 0; c < 6; c++)
    if (c == t.single) t.c1 = t.coef[c];
  return t;
}

// Whole forward spectrum from the few nonzero planes z in [lo, hi) by direct
// DFT: X(kz) = sum_z x(z) W_L^(kz z), written at the DIF positions of the tile.
template <int L>
__device__ __forceinline__ void direct_in(cx<float>* tile, const cx<float>* tw, const cx<float>* col,
                                          long long zstride, int lo, int hi, cx<float> (*mz)[TB]) {
  const int np = hi - lo;
  if (threadIdx.x < kDirectPlanes * TB) {
    const int p = threadIdx.x / TB, line = threadIdx.x % TB;
    mz[p][line] = p < np ? col[(long long)(lo + p) * zstride + line] : zero<float>();
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L * TB; i += kNT) {
    const int pos = i / TB, line = i % TB;
    const int kz = k_of_pos<L>(pos);
    cx<float> acc = zero<float>();
    for (int p = 0; p < np; p++) acc = acc + cmul(mz[p][line], tw[(kz * (lo + p)) % L]);
    tile[i] = acc;
  }
}

// Inverse transform evaluated only at the few planes z in [lo, hi):
// x(z) = sum_kz X(kz) W_L^(-kz z), from the whole spectrum in the tile.
template <int L>
__device__ __forceinline__ void direct_out(const cx<float>* tile, const cx<float>* tw, cx<float>* col,
                                           long long zstride, int lo, int hi, cx<float> (*part)[TB]) {
  constexpr int PARTS = kNT / TB;
  const int line = threadIdx.x % TB, pr = threadIdx.x / TB;
  for (int z = lo; z < hi; z++) {
    cx<float> acc = zero<float>();
    for (int pos = pr; pos < L; pos += PARTS) {
      const int kz = k_of_pos<L>(pos);
      acc = acc + cmulc(tile[pos * TB + line], tw[(kz * z) % L]);
    }
    part[pr][line] = acc;
    __syncthreads();
    if (threadIdx.x < TB) {
      cx<float> s = zero<float>();
      for (int q = 0; q < PARTS; q++) s = s + part[q][threadIdx.x];
      col[(long long)z * zstride + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// One input slot, one output per block (grid.z = output index).
template <int L>
__global__ void __launch_bounds__(kNT, 3) k_z1(ZArgs a) {
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  __shared__ cx<float> small[kNT / TB][TB];
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int chunk = blockIdx.x, o = blockIdx.z;
  const int2 col = a.zcol[blockIdx.y];  // (ky position, ky)
  const int kyf = col.y <= a.Ly / 2 ? col.y : a.Ly - col.y;
  const float sy = col.y <= a.Ly / 2 ? 1.0f : -1.0f;
  const long long colo = (long long)col.x * a.P + chunk * TB;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.buf) + a.in_slot[0] * a.cstride + colo;
  cx<float>* out = reinterpret_cast<cx<float>*>(a.buf) + a.out_slot[o] * a.cstride + colo;
  int ilo = 0, ihi = a.n_in, olo = 0, ohi = a.n_out;
  if (a.in_ext) {
    ilo = max(a.ext[0], 0);
    ihi = min(a.ext[1], a.n_in);
  }
  if (a.out_ext) {
    olo = max(a.ext[0], 0);
    ohi = min(a.ext[1], a.n_out);
  }
  ihi = max(ihi, ilo);
  ohi = max(ohi, olo);
  const bool din = ihi - ilo <= kDirectPlanes, dout = ohi - olo <= kDirectPlanes;
  const TensorCol tcol = make_tcol(a, o, 0, kyf, sy, chunk * TB);
  __syncthreads();
  if (din) {
    direct_in<L>(tile, tw, in, a.zstride, ilo, ihi, small);
  } else {
    dif_stage0_load<float, L, kNT>(tile, tw, [&](int pos, int line) {
      return (pos >= ilo && pos < ihi) ? in[pos * a.zstride + line] : zero<float>();
    });
    __syncthreads();
    DifRange<float, L, kNT, 1, S - 1>::run(tile, tw);
  }
  __syncthreads();
  {  // last forward stage, tensor product, first inverse stage (M = 1: R consecutive positions)
    using SS = StageShape<L, S - 1>;
    constexpr int R = SS::R;
    constexpr int ITER = (SS::NU + kNT - 1) / kNT;
#pragma unroll 1
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (SS::NU % kNT == 0 || u < SS::NU) {
        const int line = u % TB, g = u / TB;
        cx<float> v[R];
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = tile[(g * R + q) * TB + line];
        if (!din) Dft<float, R, false>::run(v);
        TensorCol tl = tcol;
        tl.T += line;
        const int kb = k_of_group<L>(g);
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = scale(v[q], tl.at(kb + q * (L / R), L));
        if (!dout) Dft<float, R, true>::run(v);
#pragma unroll
        for (int q = 0; q < R; q++) tile[(g * R + q) * TB + line] = v[q];
      }
    }
  }
  __syncthreads();
  if (dout) {
    direct_out<L>(tile, tw, out, a.zstride, olo, ohi, small);
  } else {
    DitRange<float, L, kNT, 1, S - 1>::run(tile, tw);
    dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
      if (pos >= olo && pos < ohi) out[pos * a.zstride + line] = v;
    });
  }
}

// One input, every output in one block, for two-stage plans with R0 = 2 R1 = 2 M0 and
// n_in, n_out <= L/2 (L = 512 = 32 x 16): the forward transform of the column tile is
// computed once. Thread (line, j) runs stage-0 unit j (the radix-32 DFT of an input
// whose upper half is zero, as two 16-point DFTs); thread (line, g) then finishes the
// last-stage units g and g + R0/2 and keeps their spectra in tensor memory (64 columns of
// its lane). For each output: the spectra times s_o (the tensor combination), the first
// inverse stage into the tile, and the last inverse stage, which forms only the rows
// z < L/2 and writes those in [olo, ohi).
// Tensor factors of last-stage unit g for output o: frequencies kz = kb + q L/R1 (kb =
// k_of_group(g)). With one tensor component the folded row of every q is a compile-time
// offset from one of two bases (kz <= L/2 for q < R1/2, above for q > R1/2, and at q = R1/2
// unless kb = 0), and the sign under kz -> L - kz is fixed per side.
template <int L>
__device__ __forceinline__ void z_factors(const TensorCol& tc, int kb, float* f) {
  constexpr int R1 = StageShape<L, plan_stages(L) - 1>::R, QS = L / R1;
  if (tc.single >= 0) {
    const int c = tc.single;
    const float* lo = tc.T + c * tc.Tc + kb * tc.Tz;
    const float* hi = tc.T + c * tc.Tc + (L - kb) * tc.Tz;
    const float slo = tc.c1 * ((c == 3 || c == 5) ? tc.sy : 1.0f);
    const float shi = (c == 4 || c == 5) ? -slo : slo;
#pragma unroll
    for (int q = 0; q < R1; q++) {
      const long long off = (long long)q * QS * tc.Tz;
      if (q < R1 / 2) f[q] = slo * lo[off];
      else if (q > R1 / 2) f[q] = shi * hi[-off];
      else f[q] = kb == 0 ? slo * lo[off] : shi * hi[-off];
    }
  } else {
#pragma unroll
    for (int q = 0; q < R1; q++) f[q] = tc.at(kb + q * QS, L);
  }
}

constexpr unsigned kZmTmemCols = 128;  // 64 per thread; two warps share each lane quarter
template <int L, bool EXT>
__global__ void __launch_bounds__(kNT, 2) k_z1m(ZArgs a) {
  using S0 = StageShape<L, 0>;
  using S1 = StageShape<L, 1>;
  constexpr int R0 = S0::R, M0 = S0::M, R1 = S1::R;
  static_assert(R0 == 2 * R1 && M0 == R1 && M0 * TB == kNT && (L / R1) * TB == 2 * kNT, "plan");
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  __shared__ unsigned tslot;
  __shared__ cx<float> small[kNT / TB][TB];
  const int t = threadIdx.x, warp = t / 32;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  if (warp == 0) {
    tmem_alloc(&tslot, kZmTmemCols);
    tmem_relinquish();
  }
  const int chunk = blockIdx.x;
  const int2 col = a.zcol[blockIdx.y];  // (ky position, ky)
  const int kyf = col.y <= a.Ly / 2 ? col.y : a.Ly - col.y;
  const float sy = col.y <= a.Ly / 2 ? 1.0f : -1.0f;
  const long long colo = (long long)col.x * a.P + chunk * TB;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.buf) + a.in_slot[0] * a.cstride + colo;
  int ilo = 0, ihi = a.n_in, olo = 0, ohi = a.n_out;
  if (a.in_ext) {
    ilo = max(a.ext[0], 0);
    ihi = min(a.ext[1], a.n_in);
  }
  if (a.out_ext) {
    olo = max(a.ext[0], 0);
    ohi = min(a.ext[1], a.n_out);
  }
  ihi = max(ihi, ilo);
  ohi = max(ohi, olo);
  // a few planes on either side: direct transforms of those planes instead
  const bool din = EXT && ihi - ilo <= kDirectPlanes, dout = EXT && ohi - olo <= kDirectPlanes;
  const int line = t % TB, j = t / TB;
  // the tensor factors of both last-stage units for output o, loaded one phase ahead of
  // their use (output 0's with the input rows)
  float f[2][R1];
  auto load_factors = [&](int o) {
    const TensorCol tcol = make_tcol(a, o, 0, kyf, sy, chunk * TB + line);
#pragma unroll
    for (int it = 0; it < 2; it++) z_factors<L>(tcol, k_of_group<L>(it * (R0 / 2) + j), f[it]);
  };
  if (din) {  // the whole spectrum at its DIF positions
    load_factors(0);
    direct_in<L>(tile, tw, in, a.zstride, ilo, ihi, small);
  } else {  // stage 0: rows z = j + q M0 < L/2 in, positions j + q M0 (q < R0) of the tile out
    cx<float> v[R0];
#pragma unroll
    for (int q = 0; q < R0 / 2; q++) {
      const int z = j + q * M0;
      v[q] = (z >= ilo && z < ihi) ? in[z * a.zstride + line] : zero<float>();
    }
    load_factors(0);
    dft32_half_input<false>(v);
    if (j != 0) {
#pragma unroll
      for (int q = 1; q < R0; q++) v[q] = cmul(v[q], tw[j * q]);
    }
#pragma unroll
    for (int q = 0; q < R0; q++) tile[(j + q * M0) * TB + line] = v[q];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tsp = tslot + ((unsigned)((warp % 4) * 32) << 16) + (unsigned)((warp / 4) * 64);
  // last forward stage of units g = t / TB and g + R0/2, spectra into tensor memory
#pragma unroll
  for (int it = 0; it < 2; it++) {
    const int g = it * (R0 / 2) + j;
    cx<float> v[R1];
#pragma unroll
    for (int q = 0; q < R1; q++) v[q] = tile[(g * R1 + q) * TB + line];
    if (!din) DftF<R1, false>::run(v);
#pragma unroll
    for (int c = 0; c < R1 / 8; c++) {
      float b[16];
#pragma unroll
      for (int k = 0; k < 8; k++) {
        b[2 * k] = v[8 * c + k].x;
        b[2 * k + 1] = v[8 * c + k].y;
      }
      tc_st16(tsp + 32 * it + 16 * c, b);
    }
  }
  tc_wait_st();
  for (int o = 0; o < a.nout; o++) {
    __syncthreads();  // every read of the tile (previous output's last stage, or the spectra) is done
#pragma unroll
    for (int it = 0; it < 2; it++) {  // spectra times s_o, first inverse stage
      const int g = it * (R0 / 2) + j;
      cx<float> v[R1];
#pragma unroll
      for (int c = 0; c < R1 / 8; c++) {
        float b[16];
        tc_ld16(tsp + 32 * it + 16 * c, b);
        tc_wait_ld();
#pragma unroll
        for (int k = 0; k < 8; k++) v[8 * c + k] = scale(mk(b[2 * k], b[2 * k + 1]), f[it][8 * c + k]);
      }
      if (!dout) DftF<R1, true>::run(v);
#pragma unroll
      for (int q = 0; q < R1; q++) tile[(g * R1 + q) * TB + line] = v[q];
    }
    if (o + 1 < a.nout) load_factors(o + 1);
    __syncthreads();
    if (dout) {  // the few output planes from the whole spectrum
      direct_out<L>(tile, tw, reinterpret_cast<cx<float>*>(a.buf) + a.out_slot[o] * a.cstride + colo, a.zstride,
                    olo, ohi, small);
    } else {  // last inverse stage: positions j + q M0 in, rows z = j + q M0 < L/2 out
      cx<float> v[R0];
#pragma unroll
      for (int q = 0; q < R0; q++) v[q] = tile[(j + q * M0) * TB + line];
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R0; q++) v[q] = cmulc(v[q], tw[j * q]);
      }
      dft_low_half<R0, true>(v);
      cx<float>* out = reinterpret_cast<cx<float>*>(a.buf) + a.out_slot[o] * a.cstride + colo;
#pragma unroll
      for (int q = 0; q < R0 / 2; q++) {
        const int z = j + q * M0;
        if (z >= olo && z < ohi) out[z * a.zstride + line] = v[q];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tslot, kZmTmemCols);
  }
}

// Several input slots: a cluster of nin blocks per (column tile, column).
template <int L>
__global__ void __launch_bounds__(kNT, 2) k_z3(ZArgs a) {
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  __shared__ cx<float> small[kNT / TB][TB];
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int chunk = blockIdx.x / a.nin;
  const int2 col = a.zcol[blockIdx.y];
  const int kyf = col.y <= a.Ly / 2 ? col.y : a.Ly - col.y;
  const float sy = col.y <= a.Ly / 2 ? 1.0f : -1.0f;
  const long long colo = (long long)col.x * a.P + chunk * TB;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.buf) + a.in_slot[r] * a.cstride + colo;
  int ilo = 0, ihi = a.n_in, olo = 0, ohi = a.n_out;
  if (a.in_ext) {
    ilo = max(a.ext[0], 0);
    ihi = min(a.ext[1], a.n_in);
  }
  if (a.out_ext) {
    olo = max(a.ext[0], 0);
    ohi = min(a.ext[1], a.n_out);
  }
  ihi = max(ihi, ilo);
  ohi = max(ohi, olo);
  const bool din = ihi - ilo <= kDirectPlanes, dout = ohi - olo <= kDirectPlanes;
  __syncthreads();
  if (din) {
    direct_in<L>(tile, tw, in, a.zstride, ilo, ihi, small);
  } else if constexpr (zmulti_plan<L>()) {  // n_in <= L/2: the half-zero radix-32 stage, then radix 16
    constexpr int R0 = StageShape<L, 0>::R, M0 = StageShape<L, 0>::M, R1 = StageShape<L, 1>::R;
    const int line = threadIdx.x % TB, j = threadIdx.x / TB;
    {
      cx<float> v[R0];
#pragma unroll
      for (int q = 0; q < R0 / 2; q++) {
        const int z = j + q * M0;
        v[q] = (z >= ilo && z < ihi) ? in[z * a.zstride + line] : zero<float>();
      }
      dft32_half_input<false>(v);
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R0; q++) v[q] = cmul(v[q], tw[j * q]);
      }
#pragma unroll
      for (int q = 0; q < R0; q++) tile[(j + q * M0) * TB + line] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 2; it++) {
      const int g = it * (R0 / 2) + j;
      cx<float> v[R1];
#pragma unroll
      for (int q = 0; q < R1; q++) v[q] = tile[(g * R1 + q) * TB + line];
      DftF<R1, false>::run(v);
#pragma unroll
      for (int q = 0; q < R1; q++) tile[(g * R1 + q) * TB + line] = v[q];
    }
  } else {
    dif_stage0_load<float, L, kNT>(tile, tw, [&](int pos, int line) {
      return (pos >= ilo && pos < ihi) ? in[pos * a.zstride + line] : zero<float>();
    });
    __syncthreads();
    DifRange<float, L, kNT, 1, S>::run(tile, tw);
  }
  cluster.sync();  // every input spectrum of the cluster is complete

  using SS = StageShape<L, S - 1>;
  constexpr int R = SS::R;
  constexpr int ITER = (SS::NU + kNT - 1) / kNT;
  cx<float> res[ITER][R];
  const bool active = r < a.nout;
  if (active) {
    const cx<float>* src[3];
    TensorCol tc[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
      src[i] = i < a.nin ? cluster.map_shared_rank(tile, i) : tile;
      if constexpr (!zmulti_plan<L>()) tc[i] = make_tcol(a, r, i < a.nin ? i : 0, kyf, sy, chunk * TB);
    }
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (SS::NU % kNT == 0 || u < SS::NU) {
        const int line = u % TB, g = u / TB;
        const int kb = k_of_group<L>(g);
        if constexpr (zmulti_plan<L>()) {
          // the factors of one input at a time, all loads in flight (two folded-row bases)
#pragma unroll
          for (int q = 0; q < R; q++) res[it][q] = zero<float>();
#pragma unroll
          for (int i = 0; i < 3; i++) {
            if (i < a.nin) {
              const TensorCol tl = make_tcol(a, r, i, kyf, sy, chunk * TB + line);  // made here: fewer live registers
              float f[R];
              z_factors<L>(tl, kb, f);
#pragma unroll
              for (int q = 0; q < R; q++) res[it][q] = res[it][q] + scale(src[i][(g * R + q) * TB + line], f[q]);
            }
          }
          if (!dout) DftF<R, true>::run(res[it]);
          if (it == 0) {  // the first unit waits in shared memory (its registers go to the second)
#pragma unroll
            for (int q = 0; q < R; q++) tile[L * TB + q * kNT + threadIdx.x] = res[0][q];
          }
        } else {
#pragma unroll
          for (int q = 0; q < R; q++) {
            const int pos = (g * R + q) * TB + line;
            const int kz = kb + q * (L / R);
            cx<float> acc = zero<float>();
#pragma unroll
            for (int i = 0; i < 3; i++) {
              if (i < a.nin) {
                TensorCol tl = tc[i];
                tl.T += line;
                acc = acc + scale(src[i][pos], tl.at(kz, L));
              }
            }
            res[it][q] = acc;
          }
          if (!dout) Dft<float, R, true>::run(res[it]);
        }
      }
    }
  }
  cluster.sync();  // all reads of remote tiles are done
  if (!active) return;
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int u = it * kNT + threadIdx.x;
    if (SS::NU % kNT == 0 || u < SS::NU) {
      const int line = u % TB, g = u / TB;
#pragma unroll
      for (int q = 0; q < R; q++)
        tile[(g * R + q) * TB + line] = (zmulti_plan<L>() && it == 0) ? tile[L * TB + q * kNT + threadIdx.x] : res[it][q];
    }
  }
  __syncthreads();
  cx<float>* out = reinterpret_cast<cx<float>*>(a.buf) + a.out_slot[r] * a.cstride + colo;
  if (dout) {
    direct_out<L>(tile, tw, out, a.zstride, olo, ohi, small);
  } else {
    if constexpr (zmulti_plan<L>()) {  // n_out <= L/2: only the rows z < L/2 are formed
      constexpr int R0 = StageShape<L, 0>::R, M0 = StageShape<L, 0>::M;
      const int line = threadIdx.x % TB, j = threadIdx.x / TB;
      cx<float> v[R0];
#pragma unroll
      for (int q = 0; q < R0; q++) v[q] = tile[(j + q * M0) * TB + line];
      if (j != 0) {
#pragma unroll
        for (int q = 1; q < R0; q++) v[q] = cmulc(v[q], tw[j * q]);
      }
      dft_low_half<R0, true>(v);
#pragma unroll
      for (int q = 0; q < R0 / 2; q++) {
        const int z = j + q * M0;
        if (z >= olo && z < ohi) out[z * a.zstride + line] = v[q];
      }
    } else {
      DitRange<float, L, kNT, 1, S - 1>::run(tile, tw);
      dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
        if (pos >= olo && pos < ohi) out[pos * a.zstride + line] = v;
      });
    }
  }
}

template <int L>
size_t tile_smem() {
  return (size_t)(L + L * TB) * sizeof(float2);
}

template <int L, bool INV>
int run_y(const YArgs& a, int ncomp, cudaStream_t s) {
  const size_t sm = tile_smem<L>();
  static bool init = false;
  if (!init) {
    if (cudaFuncSetAttribute(k_ypass<L, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init = true;
  }
  if (a.nplanes == 0 || ncomp == 0) return 0;
  dim3 grid(a.P / TB, a.nplanes, ncomp);
  return launch_k(k_ypass<L, INV>, grid, dim3(kNT), sm, s, a.pdl != 0, a) == cudaSuccess ? 0 : -1;
}

template <int L>
int run_z(const ZArgs& a, cudaStream_t s) {
  const size_t sm = tile_smem<L>();
  if constexpr (zmulti_plan<L>()) {
    if (a.nin == 1 && a.n_in <= L / 2 && a.n_out <= L / 2) {
      // EXT: the input or output planes come from the device range a.ext, and a few of them
      // take the direct transforms
      const bool ext = a.in_ext || a.out_ext;
      auto kern = ext ? k_z1m<L, true> : k_z1m<L, false>;
      static bool initm[2] = {false, false};
      if (!initm[ext]) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return -1;
        initm[ext] = true;
      }
      kern<<<dim3(a.P / TB, a.Ly), kNT, sm, s>>>(a);
      return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
    }
  }
  if (a.nin == 1) {
    static bool init = false;
    if (!init) {
      if (cudaFuncSetAttribute(k_z1<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return -1;
      init = true;
    }
    dim3 grid(a.P / TB, a.Ly, a.nout);
    k_z1<L><<<grid, kNT, sm, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
  }
  // the 32 x 16 plan keeps each thread's first output unit in shared memory beside the tile
  const size_t sm3 = sm + (zmulti_plan<L>() ? (size_t)kNT * TB * sizeof(float2) : 0);
  static bool init3 = false;
  if (!init3) {
    if (cudaFuncSetAttribute(k_z3<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3) != cudaSuccess)
      return -1;
    init3 = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.nin * (a.P / TB), a.Ly, 1);
  cfg.blockDim = dim3(kNT, 1, 1);
  cfg.dynamicSmemBytes = sm3;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.nin;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_z3<L>, a) != cudaSuccess) return -1;
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

size_t zpass_smem(int L) { return (size_t)(L + L * TB) * sizeof(float2); }

int launch_yfwd(int L, const YArgs& a, int ncomp, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_y<LL, false>(a, ncomp, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}
int launch_yinv(int L, const YArgs& a, int ncomp, cudaStream_t s) {
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_y<LL, true>(a, ncomp, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}
int launch_zpass(int L, const ZArgs& a, cudaStream_t s) {
  if (a.nin < 1 || a.nin > 3 || a.nout < 1 || a.nout > 3 || (a.nin > 1 && a.nout > a.nin)) return -2;
  switch (L) {
#define TM_CASE(LL) \
  case LL:          \
    return run_z<LL>(a, s);
    TM_FOR_EACH_L(TM_CASE)
#undef TM_CASE
  }
  return -2;
}

}  // namespace tmk
