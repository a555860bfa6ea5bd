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

namespace cg = cooperative_groups;

namespace tmk {

namespace {

template <int L, bool INV>
__global__ void __launch_bounds__(kNT, 3) k_ypass(YArgs a) {
  constexpr int S = plan_stages(L);
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int chunk = blockIdx.x, z = blockIdx.y;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.in) + a.in_slot[blockIdx.z] * a.in_cstride +
                        z * a.in_zstride + chunk * TB;
  cx<float>* out = reinterpret_cast<cx<float>*>(a.out) + a.out_slot[blockIdx.z] * a.out_cstride +
                   z * a.out_zstride + chunk * TB;
  __syncthreads();
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

// The needed unique components of N^ at (kz, ky, kx) with the parity signs of
// the folded storage applied (kx <= L/2 always, so only ky and kz flip signs).
struct TensorAt {
  const float* T;  // at (kyf, kx): T + kyf * P + kx
  long long Tc, Tz;
  __device__ __forceinline__ void load(int kzf, float sy, float sz, int need, float n[6]) const {
    const float* t = T + kzf * Tz;
    n[0] = (need & 1) ? t[0] : 0.0f;
    n[1] = (need & 2) ? t[Tc] : 0.0f;
    n[2] = (need & 4) ? t[2 * Tc] : 0.0f;
    n[3] = (need & 8) ? sy * t[3 * Tc] : 0.0f;
    n[4] = (need & 16) ? sz * t[4 * Tc] : 0.0f;
    n[5] = (need & 32) ? sy * sz * t[5 * Tc] : 0.0f;
  }
};

__device__ __forceinline__ float contract6(const float* c, const float* n) {
  return c[0] * n[0] + c[1] * n[1] + c[2] * n[2] + c[3] * n[3] + c[4] * n[4] + c[5] * n[5];
}

// One input slot, one output per block (grid.z = output index).
template <int L>
__global__ void __launch_bounds__(kNT, 3) k_z1(ZArgs a) {
  constexpr int S = plan_stages(L);
  constexpr int LH = L / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int chunk = blockIdx.x, o = blockIdx.z;
  const int2 col = a.zcol[blockIdx.y];  // (ky position, ky)
  const int kyf = col.y <= a.Ly / 2 ? col.y : a.Ly - col.y;
  const float sy = col.y <= a.Ly / 2 ? 1.0f : -1.0f;
  const long long colo = (long long)col.x * a.P + chunk * TB;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.buf) + a.in_slot[0] * a.cstride + colo;
  cx<float>* out = reinterpret_cast<cx<float>*>(a.buf) + a.out_slot[o] * a.cstride + colo;
  float coef[6];
#pragma unroll
  for (int c = 0; c < 6; c++) coef[c] = a.coef[o][0][c];
  const int need = a.need[o];
  __syncthreads();
  dif_stage0_load<float, L, kNT>(tile, tw, [&](int pos, int line) {
    return pos < a.n_in ? in[pos * a.zstride + line] : zero<float>();
  });
  __syncthreads();
  DifRange<float, L, kNT, 1, S - 1>::run(tile, tw);
  {
    using SS = StageShape<L, S - 1>;
    constexpr int R = SS::R;
    constexpr int ITER = (SS::NU + kNT - 1) / kNT;
    TensorAt ta{a.T + kyf * (long long)a.P + chunk * TB, a.Tc, a.Tz};
#pragma unroll 1
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (SS::NU % kNT == 0 || u < SS::NU) {
        const int line = u % TB, g = u / TB;
        cx<float> v[R];
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = tile[(g * R + q) * TB + line];
        Dft<float, R, false>::run(v);
        TensorAt tl = ta;
        tl.T += line;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int kz = k_of_pos<L>(g * R + q);
          const int kzf = kz <= LH ? kz : L - kz;
          const float sz = kz <= LH ? 1.0f : -1.0f;
          float n[6];
          tl.load(kzf, sy, sz, need, n);
          v[q] = scale(v[q], contract6(coef, n));
        }
        Dft<float, R, true>::run(v);
#pragma unroll
        for (int q = 0; q < R; q++) tile[(g * R + q) * TB + line] = v[q];
      }
    }
  }
  __syncthreads();
  DitRange<float, L, kNT, 1, S - 1>::run(tile, tw);
  dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
    if (pos < a.n_out) out[pos * a.zstride + line] = v;
  });
}

// Several input slots: a cluster of nin blocks per (column tile, column).
template <int L>
__global__ void __launch_bounds__(kNT, 2) k_z3(ZArgs a) {
  constexpr int S = plan_stages(L);
  constexpr int LH = L / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  cx<float>* tw = reinterpret_cast<cx<float>*>(smem);
  cx<float>* tile = tw + L;
  cg::cluster_group cluster = cg::this_cluster();
  const int r = (int)cluster.block_rank();
  load_twiddles<float, kNT>(tw, reinterpret_cast<const cx<float>*>(a.tw), L);
  const int chunk = blockIdx.x / a.nin;
  const int2 col = a.zcol[blockIdx.y];
  const int kyf = col.y <= a.Ly / 2 ? col.y : a.Ly - col.y;
  const float sy = col.y <= a.Ly / 2 ? 1.0f : -1.0f;
  const long long colo = (long long)col.x * a.P + chunk * TB;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.buf) + a.in_slot[r] * a.cstride + colo;
  __syncthreads();
  dif_stage0_load<float, L, kNT>(tile, tw, [&](int pos, int line) {
    return pos < a.n_in ? in[pos * a.zstride + line] : zero<float>();
  });
  __syncthreads();
  DifRange<float, L, kNT, 1, S>::run(tile, tw);
  cluster.sync();  // every input spectrum of the cluster is complete

  using SS = StageShape<L, S - 1>;
  constexpr int R = SS::R;
  constexpr int ITER = (SS::NU + kNT - 1) / kNT;
  cx<float> res[ITER][R];
  const bool active = r < a.nout;
  if (active) {
    const cx<float>* src[3];
#pragma unroll
    for (int i = 0; i < 3; i++) src[i] = i < a.nin ? cluster.map_shared_rank(tile, i) : tile;
    float coef[3][6];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int c = 0; c < 6; c++) coef[i][c] = a.coef[r][i][c];
    const int need = a.need[r];
    TensorAt ta{a.T + kyf * (long long)a.P + chunk * TB, a.Tc, a.Tz};
#pragma unroll
    for (int it = 0; it < ITER; it++) {
      const int u = it * kNT + threadIdx.x;
      if (SS::NU % kNT == 0 || u < SS::NU) {
        const int line = u % TB, g = u / TB;
        TensorAt tl = ta;
        tl.T += line;
#pragma unroll
        for (int q = 0; q < R; q++) {
          const int pos = (g * R + q) * TB + line;
          const int kz = k_of_pos<L>(g * R + q);
          const int kzf = kz <= LH ? kz : L - kz;
          const float sz = kz <= LH ? 1.0f : -1.0f;
          float n[6];
          tl.load(kzf, sy, sz, need, n);
          cx<float> acc = zero<float>();
#pragma unroll
          for (int i = 0; i < 3; i++) {
            if (i < a.nin) acc = acc + scale(src[i][pos], contract6(coef[i], n));
          }
          res[it][q] = acc;
        }
        Dft<float, R, true>::run(res[it]);
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
      for (int q = 0; q < R; q++) tile[(g * R + q) * TB + line] = res[it][q];
    }
  }
  __syncthreads();
  DitRange<float, L, kNT, 1, S - 1>::run(tile, tw);
  cx<float>* out = reinterpret_cast<cx<float>*>(a.buf) + a.out_slot[r] * a.cstride + colo;
  dit_stage0_store<float, L, kNT>(tile, tw, [&](int pos, int line, cx<float> v) {
    if (pos < a.n_out) out[pos * a.zstride + line] = v;
  });
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
  k_ypass<L, INV><<<grid, kNT, sm, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

template <int L>
int run_z(const ZArgs& a, cudaStream_t s) {
  const size_t sm = tile_smem<L>();
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
  static bool init3 = false;
  if (!init3) {
    if (cudaFuncSetAttribute(k_z3<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -1;
    init3 = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.nin * (a.P / TB), a.Ly, 1);
  cfg.blockDim = dim3(kNT, 1, 1);
  cfg.dynamicSmemBytes = sm;
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
