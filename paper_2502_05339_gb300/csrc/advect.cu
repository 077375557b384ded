// Density carried by the DMD velocity (Sec. 7.2): the velocity frames come
// from the model (Eq. large_time_step, reconstructed in batches by the tall
// product Phi_R C), the density is advanced through them by semi-Lagrangian
// steps on the periodic MAC grid of the snapshots:
//   rho_{k+1}(c) = rho_k(c - dt u_k(c)),
// u_k(c) the velocity at the centre of cell c (per axis the mean of the two
// faces around it; component d of a frame sits on the low d-face of each
// cell), rho_k sampled by multilinear interpolation with periodic wrap, in
// grid units.  One thread per cell; each step reads one velocity frame and
// the density once and writes the density once (HBM-bound).  Cell indices
// are 32-bit (N^dim < 2^31, checked by the caller).
#include "common.cuh"

namespace dmd {

namespace {

// i mod N for any int i; one compare-and-add in the common case |i| < 2N.
__device__ __forceinline__ int wrap(int i, int N) {
  if (i >= 0 && i < N) return i;
  if (i < 0 && i >= -N) return i + N;
  if (i >= N && i < 2 * N) return i - N;
  i %= N;
  return i < 0 ? i + N : i;
}

// i mod N for N a power of two (two's complement: negative i too).
__device__ __forceinline__ int wrap_p2(int i, int N) { return i & (N - 1); }

// Cell coordinates of cell e (C order): 32-bit unsigned divisions, or shifts
// by lgN when N is a power of two (P2).
template <int DIM, bool P2 = false>
__device__ __forceinline__ void cell_coords(unsigned e, int N, int* coord, int* stride, int lgN = 0) {
  if (P2) {
    const unsigned m = (unsigned)N - 1u;
    coord[DIM - 1] = (int)(e & m);
    stride[DIM - 1] = 1;
    if (DIM == 2) {
      coord[0] = (int)(e >> lgN);
      stride[0] = N;
    } else {
      coord[1] = (int)((e >> lgN) & m);
      coord[0] = (int)(e >> (2 * lgN));
      stride[1] = N;
      stride[0] = N * N;
    }
    return;
  }
  const unsigned row = e / (unsigned)N;
  coord[DIM - 1] = (int)(e - row * (unsigned)N);
  stride[DIM - 1] = 1;
  if (DIM == 2) {
    coord[0] = (int)row;
    stride[0] = N;
  } else {
    const unsigned i = row / (unsigned)N;
    coord[1] = (int)(row - i * (unsigned)N);
    coord[0] = (int)i;
    stride[1] = N;
    stride[0] = N * N;
  }
}

// Multilinear sample of rho at the corners lo/hi (per-axis offsets) with
// fractions f, as nested linear interpolations (last axis innermost).
template <int DIM>
__device__ __forceinline__ float sample(const float* __restrict__ rho, const int* lo, const int* hi, const float* f) {
  if (DIM == 2) {
    const float a = __ldg(rho + lo[0] + lo[1]), b = __ldg(rho + lo[0] + hi[1]);
    const float c = __ldg(rho + hi[0] + lo[1]), d = __ldg(rho + hi[0] + hi[1]);
    const float ab = fmaf(f[1], b - a, a), cd = fmaf(f[1], d - c, c);
    return fmaf(f[0], cd - ab, ab);
  } else {
    float v[2][2];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int y = 0; y < 2; ++y) {
        const int base = (x ? hi[0] : lo[0]) + (y ? hi[1] : lo[1]);
        const float a = __ldg(rho + base + lo[2]), b = __ldg(rho + base + hi[2]);
        v[x][y] = fmaf(f[2], b - a, a);
      }
    const float p0 = fmaf(f[1], v[0][1] - v[0][0], v[0][0]);
    const float p1 = fmaf(f[1], v[1][1] - v[1][0], v[1][0]);
    return fmaf(f[0], p1 - p0, p0);
  }
}

// Four consecutive cells of the last axis per thread (N % 4 == 0 and 16-byte
// aligned buffers; k_advect_sl1 otherwise): the face values come in as
// float4 rows, the coordinates are computed once for the four cells, and the
// 4 x 2^DIM density samples are independent loads in flight together (one
// cell per thread is bound by the latency of its two dependent load rounds).
// P2: N a power of two (2^lgN); coordinates and the periodic wrap become
// shifts and masks (the kernel is bound by its instruction stream).
template <int DIM, bool P2>
__global__ void __launch_bounds__(128) k_advect_sl4(int N, int lgN, const float* __restrict__ rho,
                                                    float* __restrict__ out, const float* __restrict__ u, float dt) {
  const int cells = DIM == 2 ? N * N : N * N * N;
  const unsigned f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= (unsigned)(cells / 4)) return;
  const int e0 = 4 * (int)f;
  int coord[DIM], stride[DIM];
  cell_coords<DIM, P2>((unsigned)e0, N, coord, stride, lgN);
  float cen[DIM][4];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const float* comp = u + (int64_t)d * cells;
    const float4 a = __ldg(reinterpret_cast<const float4*>(comp + e0));
    if (d == DIM - 1) {
      const float nx = __ldg(comp + (coord[d] + 4 == N ? e0 + 4 - N : e0 + 4));
      cen[d][0] = 0.5f * (a.x + a.y);
      cen[d][1] = 0.5f * (a.y + a.z);
      cen[d][2] = 0.5f * (a.z + a.w);
      cen[d][3] = 0.5f * (a.w + nx);
    } else {
      const int up = coord[d] + 1 == N ? e0 - (N - 1) * stride[d] : e0 + stride[d];
      const float4 b = __ldg(reinterpret_cast<const float4*>(comp + up));
      cen[d][0] = 0.5f * (a.x + b.x);
      cen[d][1] = 0.5f * (a.y + b.y);
      cen[d][2] = 0.5f * (a.z + b.z);
      cen[d][3] = 0.5f * (a.w + b.w);
    }
  }
  float res[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int lo[DIM], hi[DIM];
    float frac[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const float s = -dt * cen[d][c];
      const float fl = floorf(s);
      frac[d] = s - fl;
      const int b = coord[d] + (d == DIM - 1 ? c : 0) + (int)fl;
      lo[d] = (P2 ? wrap_p2(b, N) : wrap(b, N)) * stride[d];
      hi[d] = (P2 ? wrap_p2(b + 1, N) : wrap(b + 1, N)) * stride[d];
    }
    res[c] = sample<DIM>(rho, lo, hi, frac);
  }
  *reinterpret_cast<float4*>(out + e0) = make_float4(res[0], res[1], res[2], res[3]);
}

// One cell per thread (any N and alignment).
template <int DIM>
__global__ void __launch_bounds__(128) k_advect_sl1(int N, const float* __restrict__ rho, float* __restrict__ out,
                                                    const float* __restrict__ u, float dt) {
  const int cells = DIM == 2 ? N * N : N * N * N;
  const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (unsigned)cells) return;
  int coord[DIM], stride[DIM];
  cell_coords<DIM>(e, N, coord, stride);
  int lo[DIM], hi[DIM];
  float frac[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const float* comp = u + (int64_t)d * cells;
    const int up = coord[d] + 1 == N ? (int)e - (N - 1) * stride[d] : (int)e + stride[d];
    const float s = -dt * 0.5f * (__ldg(comp + e) + __ldg(comp + up));
    const float fl = floorf(s);
    frac[d] = s - fl;
    const int b = coord[d] + (int)fl;
    lo[d] = wrap(b, N) * stride[d];
    hi[d] = wrap(b + 1, N) * stride[d];
  }
  out[e] = sample<DIM>(rho, lo, hi, frac);
}

__global__ void k_iota(int32_t* out, int count, int start) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = start + i;
}

}  // namespace

dmd_status launch_advect(int dim, int N, const float* rho, float* out, const float* u, float dt, cudaStream_t st) {
  int64_t cells = N;
  for (int d = 1; d < dim; ++d) cells *= N;
  const bool vec = N % 4 == 0 && ((uintptr_t)rho & 15) == 0 && ((uintptr_t)out & 15) == 0 && ((uintptr_t)u & 15) == 0;
  if (vec) {
    const unsigned blocks = (unsigned)ceil_div(cells / 4, 128);
    int lgN = 0;
    while ((1 << lgN) < N) ++lgN;
    const bool p2 = (1 << lgN) == N;
    if (dim == 2 && p2) k_advect_sl4<2, true><<<blocks, 128, 0, st>>>(N, lgN, rho, out, u, dt);
    else if (dim == 2) k_advect_sl4<2, false><<<blocks, 128, 0, st>>>(N, lgN, rho, out, u, dt);
    else if (p2) k_advect_sl4<3, true><<<blocks, 128, 0, st>>>(N, lgN, rho, out, u, dt);
    else k_advect_sl4<3, false><<<blocks, 128, 0, st>>>(N, lgN, rho, out, u, dt);
  } else {
    const unsigned blocks = (unsigned)ceil_div(cells, 128);
    if (dim == 2) k_advect_sl1<2><<<blocks, 128, 0, st>>>(N, rho, out, u, dt);
    else k_advect_sl1<3><<<blocks, 128, 0, st>>>(N, rho, out, u, dt);
  }
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_iota(int32_t* out, int count, int start, cudaStream_t st) {
  k_iota<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(out, count, start);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

}  // namespace dmd
