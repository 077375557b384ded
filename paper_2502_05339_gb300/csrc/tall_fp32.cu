// Plain-FP32 (CUDA-core) passes over the tall snapshot matrices.
//
//  * NN: C[n x N] = A[n x Kd] * B[Kd x N]   -- sketch X Omega, power step X Z,
//    CholeskyQR step Y R^{-1}, modes X' M (Sec. 4.3, Sec. 3.1) and the
//    reconstruction Phi_R C (Eq. large_time_step).  A and C are tall
//    column-major, B is small.
//  * TN: C[Ka x N] = A^T[Ka x n] * B[n x N] -- power step X^T Q, projection
//    Q^T S and Gram matrices.  The tall dimension is split across blocks;
//    each block sums 32-row tiles in FP32, adds 32 tiles in FP32 and carries
//    the running total in FP64; the per-block FP64 partials are then added in
//    a fixed order, so the result does not depend on scheduling.
#include "common.cuh"

namespace dmd {

namespace {

constexpr int NN_BM = 128, NN_BN = 64, NN_BK = 16;

// 256 threads; thread (tx, ty) = (tid % 16, tid / 16) owns rows
// {tx*4 .. tx*4+3, 64 + tx*4 .. 64 + tx*4+3} and columns ty*4 .. ty*4+3 of the tile.
__global__ void __launch_bounds__(256) k_gemm_nn_f32(int64_t n, int Kd, int N, const float* __restrict__ A,
                                                     int64_t lda, const float* __restrict__ B,
                                                     float* __restrict__ C, int64_t ldc, int ntn) {
  __shared__ __align__(16) float As[NN_BK][NN_BM];
  __shared__ __align__(16) float Bs[NN_BK][NN_BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t bid = blockIdx.x;
  const int64_t row0 = (bid / ntn) * NN_BM;
  const int col0 = (int)(bid % ntn) * NN_BN;
  const bool full_rows = row0 + NN_BM <= n;

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  float4 ra[2];
  float rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int idx = tid + t * 256;           // 512 float4 = 16 cols x 32 float4
      const int kk = idx >> 5, r4 = (idx & 31) * 4;
      const int k = k0 + kk;
      const int64_t row = row0 + r4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < Kd) {
        const float* p = A + (int64_t)k * lda + row;
        if (full_rows) {
          v = *reinterpret_cast<const float4*>(p);
        } else {
          if (row + 0 < n) v.x = p[0];
          if (row + 1 < n) v.y = p[1];
          if (row + 2 < n) v.z = p[2];
          if (row + 3 < n) v.w = p[3];
        }
      }
      ra[t] = v;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + t * 256;             // 1024 = 64 cols x 16 k
      const int kk = e & 15, j = e >> 4;
      const int k = k0 + kk, col = col0 + j;
      rb[t] = (k < Kd && col < N) ? B[(int64_t)col * Kd + k] : 0.f;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int idx = tid + t * 256;
      const int kk = idx >> 5, r4 = (idx & 31) * 4;
      *reinterpret_cast<float4*>(&As[kk][r4]) = ra[t];
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = tid + t * 256;
      Bs[e & 15][e >> 4] = rb[t];
    }
  };

  load(0);
  for (int k0 = 0; k0 < Kd; k0 += NN_BK) {
    __syncthreads();
    store();
    __syncthreads();
    if (k0 + NN_BK < Kd) load(k0 + NN_BK);
#pragma unroll
    for (int kk = 0; kk < NN_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][64 + tx * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][ty * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
  }

#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int col = col0 + ty * 4 + j;
    if (col >= N) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t row = row0 + h * 64 + tx * 4;
      float* p = C + (int64_t)col * ldc + row;
      if (row + 3 < n) {
        *reinterpret_cast<float4*>(p) = make_float4(acc[h * 4 + 0][j], acc[h * 4 + 1][j],
                                                    acc[h * 4 + 2][j], acc[h * 4 + 3][j]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (row + i < n) p[i] = acc[h * 4 + i][j];
      }
    }
  }
}

constexpr int TN_BT = 64, TN_BR = 32, TN_PAD = 68;

// C partial for one (Ka-tile, N-tile, split): 256 threads, 4x4 outputs each.
__global__ void __launch_bounds__(256) k_gemm_tn_f32(int64_t n, int Ka, int N, const float* __restrict__ A,
                                                     int64_t lda, const float* __restrict__ B,
                                                     int64_t ldb, double* __restrict__ part,
                                                     int nta, int ntb, int64_t chunk) {
  __shared__ __align__(16) float As[TN_BR][TN_PAD];
  __shared__ __align__(16) float Bs[TN_BR][TN_PAD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int tile = blockIdx.x % (nta * ntb);
  const int split = blockIdx.x / (nta * ntb);
  const int a0 = (tile % nta) * TN_BT, b0 = (tile / nta) * TN_BT;
  const int64_t rbeg = (int64_t)split * chunk;
  const int64_t rend = min(n, rbeg + chunk);

  // three-level sum: a 32-row tile in FP32, 32 tiles in FP32, then FP64
  float acc[4][4], mid[4][4];
  double tot[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) mid[i][j] = 0.f, tot[i][j] = 0.0;

  int stretch = 0;
  for (int64_t r0 = rbeg; r0 < rend; r0 += TN_BR) {
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int idx = tid + t * 256;             // 2048 = 64 cols x 32 rows
      const int rr = idx & 31, c = idx >> 5;
      const int64_t row = r0 + rr;
      const bool rok = row < rend;
      As[rr][c] = (rok && a0 + c < Ka) ? A[(int64_t)(a0 + c) * lda + row] : 0.f;
      Bs[rr][c] = (rok && b0 + c < N) ? B[(int64_t)(b0 + c) * ldb + row] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 8
    for (int rr = 0; rr < TN_BR; ++rr) {
      const float4 a = *reinterpret_cast<const float4*>(&As[rr][tx * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[rr][ty * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) mid[i][j] += acc[i][j];
    if (++stretch == 32) {                       // 1024 rows, then fold into FP64
      stretch = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) tot[i][j] += (double)mid[i][j], mid[i][j] = 0.f;
    }
  }
  double* out = part + (int64_t)split * Ka * N;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = a0 + tx * 4 + i, b = b0 + ty * 4 + j;
      if (a < Ka && b < N) out[(int64_t)b * Ka + a] = tot[i][j] + (double)mid[i][j];
    }
}

__global__ void k_reduce_splits(int64_t count, int splits, const double* __restrict__ part,
                                double* __restrict__ C) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s = 0.0;
  for (int p = 0; p < splits; ++p) s += part[(int64_t)p * count + i];
  C[i] = s;
}

__global__ void k_f64_to_f32(int64_t count, const double* __restrict__ in, float* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) out[i] = (float)in[i];
}

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 152;
  }
  return cached;
}

}  // namespace

// Number of row splits for the TN reduction: enough blocks to fill the GPU
// about four times over, each split at least 1024 rows.
int tn_splits(int64_t n, int Ka, int N) {
  const int tiles = (int)(ceil_div(Ka, TN_BT) * ceil_div(N, TN_BT));
  int64_t want = ceil_div(4LL * 152, tiles);
  const int64_t maxs = std::max<int64_t>(1, ceil_div(n, 1024));
  if (want > maxs) want = maxs;
  if (want > 1024) want = 1024;
  return (int)std::max<int64_t>(1, want);
}

size_t tn_partial_doubles(int64_t n, int Ka, int N) {
  return (size_t)tn_splits(n, Ka, N) * Ka * N;
}

dmd_status f32_gemm_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const float* B32,
                       float* C, int64_t ldc, cudaStream_t st) {
  if (n <= 0 || N <= 0) return DMD_OK;
  const int ntn = (int)ceil_div(N, NN_BN);
  const int64_t blocks = ceil_div(n, NN_BM) * ntn;
  k_gemm_nn_f32<<<(unsigned)blocks, 256, 0, st>>>(n, Kd, N, A, lda, B32, C, ldc, ntn);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status f32_gemm_tn(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B,
                       int64_t ldb, double* C, double* part, cudaStream_t st) {
  const int splits = tn_splits(n, Ka, N);
  const int64_t chunk = round_up(ceil_div(n, splits), TN_BR);
  const int nta = (int)ceil_div(Ka, TN_BT), ntb = (int)ceil_div(N, TN_BT);
  k_gemm_tn_f32<<<(unsigned)(nta * ntb * splits), 256, 0, st>>>(n, Ka, N, A, lda, B, ldb, part,
                                                                 nta, ntb, chunk);
  DMD_LAUNCH_CHECK();
  const int64_t count = (int64_t)Ka * N;
  k_reduce_splits<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, splits, part, C);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status f64_to_f32(int64_t count, const double* in, float* out, cudaStream_t st) {
  if (count <= 0) return DMD_OK;
  k_f64_to_f32<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, in, out);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

int device_sm_count() { return sm_count(); }

}  // namespace dmd
