// Direct z convolution in (kx, ky, z) space for targets that occupy a few planes.
//
// After the x and y transforms the convolution of Sec. "Discretization",
// Eq. (convolution) is, per column (kx, ky), a 1-D convolution along z with the
// tensor transformed along x and y only:
//     out_o(z) = sum_{z'} sum_i s_oi(z - z') in_i(z'),   s_oi = v_o^T N~(z - z') u_i.
// When the outputs (forward field on the target planes) or the inputs (adjoint
// source on the target planes) occupy at most a few planes, summing this
// directly costs a few multiply-adds per complex value streamed from memory,
// instead of a forward and an inverse z FFT. The result is the same
// convolution (no approximation). Columns are read with consecutive threads on
// consecutive kx.
#include "fft.cuh"
#include "internal.h"

namespace tmk {

namespace {

// s = a - i b for one (o, i) pair at offset dz: a from the real components
// (xx, yy, zz, xy), b from the imaginary ones (xz, yz: stored r with N~ = -i r).
struct ZTensor {
  const float* T;  // Tz + kyf * P + kx
  long long Tc, Tdz;
  float sy;
  __device__ __forceinline__ void at(int dz, const float* coef, int need, float& a, float& b) const {
    const int adz = dz < 0 ? -dz : dz;
    const float sz = dz < 0 ? -1.0f : 1.0f;
    const float* t = T + adz * Tdz;
    a = 0.0f;
    b = 0.0f;
    if (need & 1) a += coef[0] * t[0];
    if (need & 2) a += coef[1] * t[Tc];
    if (need & 4) a += coef[2] * t[2 * Tc];
    if (need & 8) a += coef[3] * sy * t[3 * Tc];
    if (need & 16) b += coef[4] * sz * t[4 * Tc];
    if (need & 32) b += coef[5] * sy * sz * t[5 * Tc];
  }
};

__device__ __forceinline__ cx<float> apply_s(cx<float> v, float a, float b) {
  // (a - i b) v
  return mk(a * v.x + b * v.y, a * v.y - b * v.x);
}

// One input, one output, one tensor component (the common case: constant M0 and
// one weighted field component, or an axis-aligned M0): per streamed value one
// load, one tensor load and one complex multiply-add, with running pointers.
// c: the component; its coefficient and the column's sign are folded into `scale`.
__global__ void __launch_bounds__(256) k_zdir_simple(ZDirArgs a, int c) {
  // 32 kx x 2 columns x 4 z quarters per block
  constexpr int ZS = 4;
  const int kx = blockIdx.x * 32 + (threadIdx.x & 31);
  const int part = (threadIdx.x >> 5) & (ZS - 1);
  const int zc = blockIdx.y * 2 + (threadIdx.x >> 7);
  __shared__ cx<float> red[2][ZS][32];
  const bool valid = kx < a.P && zc < a.Ly;
  const int2 col = valid ? a.zcol[zc] : make_int2(0, 0);
  const bool lo = col.y <= a.Ly / 2;
  const int kyf = lo ? col.y : a.Ly - col.y;
  const bool imag = c >= 4;   // xz, yz: N~ = -i r
  const bool odd_z = c >= 4;  // xz, yz change sign with dz
  float scale = a.coef[0][0][c];
  if ((c == 3 || c == 5) && !lo) scale = -scale;  // odd in y
  const float* t = a.Tz + c * a.Tc + kyf * (long long)a.P + kx;
  const long long colo = (long long)col.x * a.P + kx;
  const cx<float>* in = reinterpret_cast<const cx<float>*>(a.buf) + a.in_slot[0] * a.cstride + colo;
  cx<float>* out = reinterpret_cast<cx<float>*>(a.buf) + a.out_slot[0] * a.cstride + colo;
  auto fac = [&](int dz) {
    const int adz = dz < 0 ? -dz : dz;
    float v = scale * t[adz * a.Tdz];
    if (odd_z && dz < 0) v = -v;
    return v;
  };
  if (a.nzout == 1) {  // stream the inputs onto one output plane; quarters summed in order
    const int zo = a.zout0;
    const int per = (a.nzin + ZS - 1) / ZS;
    const int z0 = a.zin0 + part * per, z1 = min(z0 + per, a.zin0 + a.nzin);
    float ar = 0.0f, ai = 0.0f;
    if (valid) {
      const cx<float>* ip = in + (long long)z0 * a.zstride;
#pragma unroll 8
      for (int z = z0; z < z1; z++) {
        const cx<float> v = *ip;
        ip += a.zstride;
        const float f = fac(zo - z);
        if (imag) {  // (-i f) v
          ar += f * v.y;
          ai -= f * v.x;
        } else {
          ar += f * v.x;
          ai += f * v.y;
        }
      }
    }
    red[threadIdx.x >> 7][part][threadIdx.x & 31] = mk(ar, ai);
    __syncthreads();
    if (part == 0 && valid) {
      cx<float> s = red[threadIdx.x >> 7][0][threadIdx.x & 31];
      for (int q = 1; q < ZS; q++) s = s + red[threadIdx.x >> 7][q][threadIdx.x & 31];
      out[(long long)zo * a.zstride] = s;
    }
  } else {  // one input plane streamed onto every output plane; quarters of the planes
    if (!valid) return;
    const int zi = a.zin0;
    const cx<float> v = in[(long long)zi * a.zstride];
    const int per = (a.nzout + ZS - 1) / ZS;
    const int z0 = a.zout0 + part * per, z1 = min(z0 + per, a.zout0 + a.nzout);
    cx<float>* op = out + (long long)z0 * a.zstride;
#pragma unroll 8
    for (int z = z0; z < z1; z++) {
      const float f = fac(z - zi);
      *op = imag ? mk(f * v.y, -f * v.x) : mk(f * v.x, f * v.y);
      op += a.zstride;
    }
  }
}


// Three inputs, three outputs with coefficients v_o = e_o, u_i = e_i (a spatially
// varying M0: the magnetization enters and the field leaves component by component):
// s_oi is the tensor component (o, i) itself, so per streamed column value the six
// components are loaded once and out_o = sum_i N_oi in_i, with N_xz = -i b4 and
// N_yz = -i b5 (odd in z; xy and yz odd in y). Same 4-way z split as k_zdir_simple.
__device__ __forceinline__ void apply_n(const cx<float> in[3], const float t[6], cx<float> out[3]) {
  // (-i b) v = (b v.y, -b v.x)
  out[0] = mk(t[0] * in[0].x + t[3] * in[1].x + t[4] * in[2].y, t[0] * in[0].y + t[3] * in[1].y - t[4] * in[2].x);
  out[1] = mk(t[3] * in[0].x + t[1] * in[1].x + t[5] * in[2].y, t[3] * in[0].y + t[1] * in[1].y - t[5] * in[2].x);
  out[2] = mk(t[4] * in[0].y + t[5] * in[1].y + t[2] * in[2].x, -t[4] * in[0].x - t[5] * in[1].x + t[2] * in[2].y);
}

__global__ void __launch_bounds__(256) k_zdir_id(ZDirArgs a) {
  constexpr int ZS = 4;
  const int kx = blockIdx.x * 32 + (threadIdx.x & 31);
  const int part = (threadIdx.x >> 5) & (ZS - 1);
  const int zc = blockIdx.y * 2 + (threadIdx.x >> 7);
  __shared__ cx<float> red[2][ZS][3][32];
  const bool valid = kx < a.P && zc < a.Ly;
  const int2 col = valid ? a.zcol[zc] : make_int2(0, 0);
  const bool lo = col.y <= a.Ly / 2;
  const int kyf = lo ? col.y : a.Ly - col.y;
  const float sy = lo ? 1.0f : -1.0f;
  const float* t0 = a.Tz + kyf * (long long)a.P + kx;
  const long long colo = (long long)col.x * a.P + kx;
  const cx<float>* buf = reinterpret_cast<const cx<float>*>(a.buf);
  cx<float>* obuf = reinterpret_cast<cx<float>*>(a.buf);
  auto tensor = [&](int dz, float t[6]) {
    const int adz = dz < 0 ? -dz : dz;
    const float sz = dz < 0 ? -1.0f : 1.0f;
    const float* p = t0 + adz * a.Tdz;
#pragma unroll
    for (int c = 0; c < 6; c++) t[c] = p[c * a.Tc];
    t[3] *= sy;
    t[4] *= sz;
    t[5] *= sy * sz;
  };
  if (a.nzout == 1) {  // stream the inputs onto one output plane; quarters summed in order
    const int zo = a.zout0;
    const int per = (a.nzin + ZS - 1) / ZS;
    const int z0 = a.zin0 + part * per, z1 = min(z0 + per, a.zin0 + a.nzin);
    cx<float> acc[3] = {zero<float>(), zero<float>(), zero<float>()};
    if (valid) {
#pragma unroll 4
      for (int z = z0; z < z1; z++) {
        cx<float> in[3];
#pragma unroll
        for (int i = 0; i < 3; i++) in[i] = buf[a.in_slot[i] * a.cstride + z * a.zstride + colo];
        float t[6];
        tensor(zo - z, t);
        cx<float> o[3];
        apply_n(in, t, o);
#pragma unroll
        for (int k = 0; k < 3; k++) acc[k] = acc[k] + o[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; k++) red[threadIdx.x >> 7][part][k][threadIdx.x & 31] = acc[k];
    __syncthreads();
    if (part == 0 && valid) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        cx<float> sum = red[threadIdx.x >> 7][0][k][threadIdx.x & 31];
        for (int q = 1; q < ZS; q++) sum = sum + red[threadIdx.x >> 7][q][k][threadIdx.x & 31];
        obuf[a.out_slot[k] * a.cstride + zo * a.zstride + colo] = sum;
      }
    }
  } else {  // one input plane onto every output plane; quarters of the planes
    if (!valid) return;
    const int zi = a.zin0;
    cx<float> in[3];
#pragma unroll
    for (int i = 0; i < 3; i++) in[i] = buf[a.in_slot[i] * a.cstride + zi * a.zstride + colo];
    const int per = (a.nzout + ZS - 1) / ZS;
    const int z0 = a.zout0 + part * per, z1 = min(z0 + per, a.zout0 + a.nzout);
#pragma unroll 4
    for (int z = z0; z < z1; z++) {
      float t[6];
      tensor(z - zi, t);
      cx<float> o[3];
      apply_n(in, t, o);
#pragma unroll
      for (int k = 0; k < 3; k++) obuf[a.out_slot[k] * a.cstride + z * a.zstride + colo] = o[k];
    }
  }
}

template <int NP>
__global__ void __launch_bounds__(256) k_zdir(ZDirArgs a) {
  const int kx = blockIdx.x * 32 + (threadIdx.x & 31);
  const int zc = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (kx >= a.P || zc >= a.Ly) return;
  const int2 col = a.zcol[zc];
  const int kyf = col.y <= a.Ly / 2 ? col.y : a.Ly - col.y;
  ZTensor zt{a.Tz + kyf * (long long)a.P + kx, a.Tc, a.Tdz, col.y <= a.Ly / 2 ? 1.0f : -1.0f};
  const long long colo = (long long)col.x * a.P + kx;
  const cx<float>* buf = reinterpret_cast<const cx<float>*>(a.buf);
  cx<float>* obuf = reinterpret_cast<cx<float>*>(a.buf);

  if (a.nzout <= a.nzin) {  // few outputs: stream the inputs, keep NP x nout sums
    cx<float> acc[3][NP];
#pragma unroll
    for (int o = 0; o < 3; o++)
#pragma unroll
      for (int p = 0; p < NP; p++) acc[o][p] = zero<float>();
#pragma unroll 8
    for (int z = a.zin0; z < a.zin0 + a.nzin; z++) {
      cx<float> in[3];
#pragma unroll
      for (int i = 0; i < 3; i++)
        if (i < a.nin) in[i] = buf[a.in_slot[i] * a.cstride + z * a.zstride + colo];
#pragma unroll
      for (int p = 0; p < NP; p++) {
        if (p >= a.nzout) break;
        const int dz = a.zout0 + p - z;
#pragma unroll
        for (int o = 0; o < 3; o++) {
          if (o >= a.nout) break;
#pragma unroll
          for (int i = 0; i < 3; i++) {
            if (i >= a.nin) break;
            float sa, sb;
            zt.at(dz, a.coef[o][i], a.need[o][i], sa, sb);
            acc[o][p] = acc[o][p] + apply_s(in[i], sa, sb);
          }
        }
      }
    }
#pragma unroll
    for (int p = 0; p < NP; p++) {
      if (p >= a.nzout) break;
#pragma unroll
      for (int o = 0; o < 3; o++)
        if (o < a.nout) obuf[a.out_slot[o] * a.cstride + (a.zout0 + p) * a.zstride + colo] = acc[o][p];
    }
  } else {  // few inputs: keep them, stream the outputs
    cx<float> in[3][NP];
#pragma unroll
    for (int p = 0; p < NP; p++)
#pragma unroll
      for (int i = 0; i < 3; i++)
        in[i][p] = (p < a.nzin && i < a.nin) ? buf[a.in_slot[i] * a.cstride + (a.zin0 + p) * a.zstride + colo]
                                               : zero<float>();
#pragma unroll 8
    for (int z = a.zout0; z < a.zout0 + a.nzout; z++) {
      cx<float> acc[3] = {zero<float>(), zero<float>(), zero<float>()};
#pragma unroll
      for (int p = 0; p < NP; p++) {
        if (p >= a.nzin) break;
        const int dz = z - (a.zin0 + p);
#pragma unroll
        for (int o = 0; o < 3; o++) {
          if (o >= a.nout) break;
#pragma unroll
          for (int i = 0; i < 3; i++) {
            if (i >= a.nin) break;
            float sa, sb;
            zt.at(dz, a.coef[o][i], a.need[o][i], sa, sb);
            acc[o] = acc[o] + apply_s(in[i][p], sa, sb);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < 3; o++)
        if (o < a.nout) obuf[a.out_slot[o] * a.cstride + z * a.zstride + colo] = acc[o];
    }
  }
}

}  // namespace

int launch_zdir(const ZDirArgs& a, cudaStream_t s) {
  const int small = a.nzout <= a.nzin ? a.nzout : a.nzin;
  if (small < 0 || small > kDirectPlanesMax) return -2;
  if (small == 0) return 0;
  dim3 grid((a.P + 31) / 32, (a.Ly + 7) / 8);
  if (a.nin == 3 && a.nout == 3 && small == 1) {  // coefficients e_o^T N e_i: each the component (o, i)
    bool id = true;
    for (int o = 0; o < 3; o++)
      for (int i = 0; i < 3; i++) {
        const int c = o == i ? o : (o + i == 1 ? 3 : (o + i == 2 ? 4 : 5));
        id = id && a.need[o][i] == (1 << c) && a.coef[o][i][c] == 1.0f;
      }
    if (id) {
      k_zdir_id<<<dim3((a.P + 31) / 32, (a.Ly + 1) / 2), 256, 0, s>>>(a);
      return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
    }
  }
  if (a.nin == 1 && a.nout == 1 && small == 1) {
    const int need = a.need[0][0];
    if (need != 0 && (need & (need - 1)) == 0) {
      k_zdir_simple<<<dim3((a.P + 31) / 32, (a.Ly + 1) / 2), 256, 0, s>>>(a, __builtin_ctz(need));
      return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
    }
  }
  if (small == 1)
    k_zdir<1><<<grid, 256, 0, s>>>(a);
  else if (small == 2)
    k_zdir<2><<<grid, 256, 0, s>>>(a);
  else if (small <= 4)
    k_zdir<4><<<grid, 256, 0, s>>>(a);
  else
    k_zdir<kDirectPlanesMax><<<grid, 256, 0, s>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace tmk
