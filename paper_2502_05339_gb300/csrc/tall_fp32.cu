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
#include "ptx.cuh"

namespace dmd {

namespace {

constexpr int NN_BM = 128, NN_BN = 64, NN_BK = 16;

// 256 threads; thread (tx, ty) = (tid % 16, tid / 16) owns rows
// {tx*4 .. tx*4+3, 64 + tx*4 .. 64 + tx*4+3} and columns ty*4 .. ty*4+3 of the tile.
__global__ void __launch_bounds__(256) k_gemm_nn_f32(int64_t n, int Kd, int N, const float* __restrict__ A,
                                                     int64_t lda, const float* __restrict__ B,
                                                     float* __restrict__ C, int64_t ldc, int ntn,
                                                     const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
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

constexpr int TN_BT = 64, TN_BR = 32, TN_STAGES = 4, TN_THREADS = 128;
constexpr uint32_t TN_BOX_BYTES = TN_BT * TN_BR * 4;        // one 32-row x 64-column box: 8 KB
constexpr uint32_t TN_STAGE_BYTES = 2 * TN_BOX_BYTES;        // A and B boxes
constexpr size_t TN_SMEM = 1024 + TN_STAGES * TN_STAGE_BYTES + 128;

// Upper-triangle tile t of an nt x nt tile grid -> (ti, tj), ti <= tj.
__device__ __forceinline__ void sym_tile(int t, int nt, int& ti, int& tj) {
  ti = 0;
  while (t >= nt - ti) {
    t -= nt - ti;
    ++ti;
  }
  tj = ti + t;
}

// Float4 of rows 4q..4q+3 of box column c in a 128-byte-swizzled box
// (each column is one 128-byte line; its 16-byte chunks are XOR-permuted by
// the line index mod 8, which makes the column-strided reads conflict-free).
__device__ __forceinline__ float4 box_ld4(const uint8_t* box, int c, int q) {
  return *reinterpret_cast<const float4*>(box + c * 128 + ((q ^ (c & 7)) << 4));
}

// Partial C = A^T B of one (64 x 64 tile, row split).  A box column c is
// A[:, a0 + c] over 32 consecutive rows; TMA streams the boxes through a
// 4-stage ring.  128 threads: warp w owns tile columns 16w .. 16w+15 (and
// skips its work where they are all past N); lane (ta, tb) = (lane % 16,
// lane / 16) owns the outputs (a0 + ta + 16 i, b0 + 16 w + tb + 2 j),
// i < 4, j < 8.  Sums: 32 rows in FP32 (acc), 32 such tiles in FP32 (mid),
// then FP64 in the per-split partial, which this CTA owns alone.  With
// sym != 0 (A = B) only tiles ti <= tj are formed.
__global__ void __launch_bounds__(TN_THREADS, 3)
    k_gemm_tn_f32(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n, int Ka,
                  int N, double* __restrict__ part, int nta, int ntb, int ntiles, int sym, int64_t chunk,
                  int32_t* err, const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;   // every CTA, before any barrier
  extern __shared__ uint8_t smraw[];
  // 1024-byte alignment by pointer arithmetic keeps the shared address space
  uint8_t* sm = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + TN_STAGES * TN_STAGE_BYTES);
  uint64_t* empty = full + TN_STAGES;
  int* abort_flag = reinterpret_cast<int*>(empty + TN_STAGES);

  const int tile = blockIdx.x % ntiles;
  const int split = blockIdx.x / ntiles;
  int ti, tj;
  if (sym) {
    sym_tile(tile, nta, ti, tj);
  } else {
    ti = tile % nta;
    tj = tile / nta;
  }
  const int a0 = ti * TN_BT, b0 = tj * TN_BT;
  const int64_t rbeg = (int64_t)split * chunk;
  const int64_t rend = min(n, rbeg + chunk);
  const int nq = rbeg < rend ? (int)((rend - rbeg + TN_BR - 1) / TN_BR) : 0;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ta = lane & 15, tb = lane >> 4;
  const bool active = b0 + 16 * warp < N;

  if (tid == 0) {
    for (int i = 0; i < TN_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], TN_THREADS / 32);   // one arrival per warp
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();

  // Thread 0 keeps up to TN_STAGES boxes in flight; a stage is refilled once
  // every warp has released it.  Before warp 0 waits for box q, box q must
  // have been issued, which needs only box q - TN_STAGES released (long done
  // in the steady state): that wait blocks.  Later boxes are issued when
  // their stages are already free, without waiting, so warp 0 is not held to
  // the pace of the slowest warp on the box it has just finished.
  int issued = 0;
  auto produce = [&](int upto, bool block) -> bool {
    for (; issued < min(nq, upto); ++issued) {
      const int s = issued % TN_STAGES;
      if (issued >= TN_STAGES) {
        const uint32_t par = (uint32_t)(issued / TN_STAGES - 1) & 1u;
        if (!block) {
          if (!mbar_test(&empty[s], par)) return true;   // not free yet: try on a later box
        } else if (!mbar_wait(&empty[s], par, abort_flag)) {
          return false;
        }
      }
      uint8_t* buf = sm + s * TN_STAGE_BYTES;
      mbar_expect_tx(&full[s], TN_STAGE_BYTES);
      const int x = (int)(rbeg + (int64_t)issued * TN_BR);
      tma_load_2d(buf, &tmA, &full[s], x, a0);
      tma_load_2d(buf + TN_BOX_BYTES, &tmB, &full[s], x, b0);
    }
    return true;
  };

  float acc[4][8], mid[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) mid[i][j] = 0.f;
  double* out = part + (int64_t)split * Ka * N;
  bool first = true;
  auto flush = [&]() {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = b0 + 16 * warp + tb + 2 * j;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int a = a0 + ta + 16 * i;
        if (a < Ka && b < N) {
          double* o = out + (int64_t)b * Ka + a;
          *o = first ? (double)mid[i][j] : *o + (double)mid[i][j];
        }
        mid[i][j] = 0.f;
      }
    }
    first = false;
  };

  // Shared-memory byte offsets of this thread's float4 loads (box_ld4 with
  // the per-thread part folded in): A column ta + 16 i has (c & 7) = ta & 7,
  // so its row-chunk k lands at ((k ^ (ta & 7)) << 4) in all four columns; B
  // column 16 w + tb + 2 j has (c & 7) = tb + 2j mod 8, whose chunk offset is
  // ((k ^ (2j mod 8)) << 4) XOR (tb << 4) = that + 16 tb when k is even and
  // - 16 tb when k is odd.  With the k loop unrolled the loads then need no
  // address arithmetic beyond an immediate offset.
  const int ta7 = ta & 7;
  const int colB = 16 * warp + tb;
  const int tbs = 16 * tb;

  int stretch = 0;
  for (int q = 0; q < nq; ++q) {
    bool ok = true;
    if (tid == 0) ok = produce(q + 1, true) && produce(q + TN_STAGES, false);
    const int s = q % TN_STAGES;
    ok = ok && mbar_wait(&full[s], (uint32_t)(q / TN_STAGES) & 1u, abort_flag);
    if (!__all_sync(0xffffffffu, ok)) break;
    if (active) {
      const uint8_t* Ab = sm + s * TN_STAGE_BYTES;
      const uint8_t* Bb = Ab + TN_BOX_BYTES;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
      const uint8_t* At = Ab + ta * 128;
      const uint8_t* Bt = Bb + colB * 128;
#pragma unroll
      for (int kq = 0; kq < TN_BR / 4; ++kq) {
        float4 av[4], bv[8];
        const uint8_t* Ak = At + ((kq ^ ta7) << 4);
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4*>(Ak + i * 16 * 128);
        const uint8_t* Bk = Bt + ((kq & 1) ? -tbs : tbs);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          bv[j] = *reinterpret_cast<const float4*>(Bk + 2 * j * 128 + ((kq ^ ((2 * j) & 7)) << 4));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            acc[i][j] = fmaf(av[i].x, bv[j].x, acc[i][j]);
            acc[i][j] = fmaf(av[i].y, bv[j].y, acc[i][j]);
            acc[i][j] = fmaf(av[i].z, bv[j].z, acc[i][j]);
            acc[i][j] = fmaf(av[i].w, bv[j].w, acc[i][j]);
          }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
    if (active) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) mid[i][j] += acc[i][j];
      if (++stretch == 32) {   // 1024 rows, then fold into FP64
        stretch = 0;
        flush();
      }
    }
  }
  if (active && (stretch > 0 || first)) flush();
  // on an abort, let the loads still in flight land before the CTA exits
  if (tid == 0 && *reinterpret_cast<volatile int*>(abort_flag)) {
    for (int q = max(0, issued - TN_STAGES); q < issued; ++q)
      mbar_wait_drain(&full[q % TN_STAGES], (uint32_t)(q / TN_STAGES) & 1u);
    raise_status(err, DMD_ETIMEOUT, 8101);
  }
}

// C = sum over splits, in split order.  With sym, entries below the diagonal
// tiles come from their mirror.
__global__ void k_reduce_splits(int Ka, int N, int splits, const double* __restrict__ part, double* __restrict__ C,
                                int sym, const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t count = (int64_t)Ka * N;
  if (i >= count) return;
  int a = (int)(i % Ka), b = (int)(i / Ka);
  if (sym && a / TN_BT > b / TN_BT) {
    const int t = a;
    a = b;
    b = t;
  }
  const int64_t src = (int64_t)b * Ka + a;
  double s = 0.0;
  for (int p = 0; p < splits; ++p) s += part[(int64_t)p * count + src];
  C[i] = s;
}

__global__ void k_f64_to_f32(int64_t count, const double* __restrict__ in, float* __restrict__ out,
                             const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) out[i] = (float)in[i];
}

// ------------------------------------------------- symmetric Gram, one read

// Symmetric Gram C = A^T A of a tall A with at most 8 * GR_MAXNS columns,
// every CTA forming the whole upper triangle of its row chunk from one read
// of that chunk (the 64 x 64 tiles of k_gemm_tn_f32 re-read A once per tile
// and form ~1.4x the distinct entries of a 201-column Gram).  The Ka columns
// are dealt into NS = ceil(Ka / 8) strided sets, set I = {I, I + NS, ...,
// I + 7 NS}; thread t owns the 8 x 8 block of set pair (I, J), I <= J, the
// t-th in row order (NS (NS + 1) / 2 <= 351 blocks; the sets are strided so
// that the 128-byte swizzle spreads a warp's loads over the banks).  Per
// 32-row stage (TMA box {32 rows, 8 NS columns}, 128-byte swizzle, columns
// past Ka zero-filled) a thread forms its 64 partial dot products in FP32
// (acc, registers, the block in two 8 x 4 halves; packed two-lane FMAs,
// even and odd rows apart), adds them into FP32 sums over 32 stages (mid,
// 1024 rows; in shared memory, element e of thread t at e * GR_THREADS + t),
// then into this CTA's FP64 partial, which it alone writes: the accuracy
// scheme of k_gemm_tn_f32.  Entry (a, b) of the upper triangle lands at
// part[cta][min(a, b) + max(a, b) Ka]; a diagonal block's entries below its
// diagonal are its duplicates and are not written.
constexpr int GR_THREADS = 352, GR_MAXNS = 26, GR_STAGES = 4, GR_BR = 32;

// c += a * b on two FP32 lanes at once (one packed FMA instruction, each
// lane rounded as a single fma.rn.f32).
__device__ __forceinline__ void ffma2(float2& c, float2 a, float2 b) {
  uint64_t cc = *reinterpret_cast<uint64_t*>(&c);
  asm("fma.rn.f32x2 %0, %1, %2, %0;"
      : "+l"(cc)
      : "l"(*reinterpret_cast<uint64_t*>(&a)), "l"(*reinterpret_cast<uint64_t*>(&b)));
  c = *reinterpret_cast<float2*>(&cc);
}

__device__ __forceinline__ void gram_pair(int t, int ns, int& I, int& J) {
  I = 0;
  while (t >= ns - I) {
    t -= ns - I;
    ++I;
  }
  J = I + t;
}

// Fold a thread's FP32 sums over 1024 rows into the CTA's FP64 partial (out
// of line: it would otherwise hold registers across the stage loop).
__device__ __noinline__ void gram_flush(float* mid, double* out, int I, int J, int ns, int Ka, int tid, bool first) {
  for (int i = 0; i < 8; ++i) {
    const int a = I + ns * i;
    for (int j = 0; j < 8; ++j) {
      const int b = J + ns * j;
      float* mp = mid + (i * 8 + j) * GR_THREADS + tid;
      if (a < Ka && b < Ka && (I != J || a <= b)) {
        double* o = out + (int64_t)max(a, b) * Ka + min(a, b);
        *o = first ? (double)*mp : *o + (double)*mp;
      }
      *mp = 0.f;
    }
  }
}

__global__ void __launch_bounds__(GR_THREADS, 1)
    k_gram_f32(const __grid_constant__ CUtensorMap tmA, int64_t n, int Ka, int ns, double* __restrict__ part,
               int64_t chunk, int32_t* err, const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;   // every CTA, before any barrier
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const uint32_t box = (uint32_t)GR_BR * 4u * 8u * (uint32_t)ns;   // bytes of one stage
  float* mid = reinterpret_cast<float*>(sm + GR_STAGES * box);   // [64][GR_THREADS]
  uint64_t* full = reinterpret_cast<uint64_t*>(mid + 64 * GR_THREADS);
  uint64_t* empty = full + GR_STAGES;
  int* abort_flag = reinterpret_cast<int*>(empty + GR_STAGES);
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr int kWarps = GR_THREADS / 32;
  const int nblk = ns * (ns + 1) / 2;
  const bool active = tid < nblk;
  int I = 0, J = 0;
  if (active) gram_pair(tid, ns, I, J);
  const int64_t rbeg = (int64_t)blockIdx.x * chunk;
  const int64_t rend = min(n, rbeg + chunk);
  const int nq = rbeg < rend ? (int)((rend - rbeg + GR_BR - 1) / GR_BR) : 0;
  if (tid == 0) {
    for (int i = 0; i < GR_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kWarps);
    }
    *abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();

  // thread 0 keeps up to GR_STAGES boxes in flight (as in k_gemm_tn_f32)
  int issued = 0;
  auto produce = [&](int upto, bool block) -> bool {
    for (; issued < min(nq, upto); ++issued) {
      const int s = issued % GR_STAGES;
      if (issued >= GR_STAGES) {
        const uint32_t par = (uint32_t)(issued / GR_STAGES - 1) & 1u;
        if (!block) {
          if (!mbar_test(&empty[s], par)) return true;
        } else if (!mbar_wait(&empty[s], par, abort_flag)) {
          return false;
        }
      }
      mbar_expect_tx(&full[s], box);
      tma_load_2d(sm + s * box, &tmA, &full[s], (int)(rbeg + (int64_t)issued * GR_BR), 0);
    }
    return true;
  };

  for (int e = 0; e < 64; ++e) mid[e * GR_THREADS + tid] = 0.f;
  double* out = part + (int64_t)blockIdx.x * Ka * Ka;
  bool first = true;
  auto flush = [&]() {
    gram_flush(mid, out, I, J, ns, Ka, tid, first);
    first = false;
  };

  int stretch = 0;
  for (int qq = 0; qq < nq; ++qq) {
    bool ok = true;
    if (tid == 0) ok = produce(qq + 1, true) && produce(qq + GR_STAGES, false);
    const int s = qq % GR_STAGES;
    ok = ok && mbar_wait(&full[s], (uint32_t)(qq / GR_STAGES) & 1u, abort_flag);
    if (!__all_sync(0xffffffffu, ok)) break;
    if (active) {
      const uint8_t* bx = sm + s * box;
      // the 8 x 8 block in two 8 x 4 halves (registers): 32 rows each.  The
      // byte offset of rows 4 q .. 4 q + 3 of column c is pre(c) ^ (16 q),
      // pre(c) = 128 c | 16 (c & 7): the 128-byte swizzle as one XOR
      uint32_t pa[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t c = (uint32_t)(I + ns * i);
        pa[i] = (c << 7) | ((c & 7u) << 4);
      }
#pragma unroll 1
      for (int jh = 0; jh < 2; ++jh) {
        uint32_t pb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t c = (uint32_t)(J + ns * (4 * jh + j));
          pb[j] = (c << 7) | ((c & 7u) << 4);
        }
        // two partial sums per entry (even and odd rows), formed by packed
        // FMAs on the (x, y) and (z, w) halves of the 4-row chunks
        float2 acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int q = 0; q < GR_BR / 4; ++q) {
          float4 bv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) bv[j] = *reinterpret_cast<const float4*>(bx + (pb[j] ^ (uint32_t)(q << 4)));
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float4 av = *reinterpret_cast<const float4*>(bx + (pa[i] ^ (uint32_t)(q << 4)));
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              ffma2(acc[i][j], make_float2(av.x, av.y), make_float2(bv[j].x, bv[j].y));
              ffma2(acc[i][j], make_float2(av.z, av.w), make_float2(bv[j].z, bv[j].w));
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) mid[(i * 8 + 4 * jh + j) * GR_THREADS + tid] += acc[i][j].x + acc[i][j].y;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
    if (active && ++stretch == 32) {   // 1024 rows, then fold into FP64
      stretch = 0;
      flush();
    }
  }
  if (active && (stretch > 0 || first)) flush();
  // on an abort, let the loads still in flight land before the CTA exits
  if (tid == 0 && *reinterpret_cast<volatile int*>(abort_flag)) {
    for (int q = max(0, issued - GR_STAGES); q < issued; ++q)
      mbar_wait_drain(&full[q % GR_STAGES], (uint32_t)(q / GR_STAGES) & 1u);
    raise_status(err, DMD_ETIMEOUT, 8102);
  }
}

// C[a, b] = C[b, a] = sum over CTAs (fixed order) of part[cta][min + max Ka].
__global__ void k_reduce_gram(int Ka, int parts, const double* __restrict__ part, double* __restrict__ C,
                              const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t count = (int64_t)Ka * Ka;
  if (i >= count) return;
  const int a = (int)(i % Ka), b = (int)(i / Ka);
  const int64_t src = (int64_t)max(a, b) * Ka + min(a, b);
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += part[(int64_t)p * count + src];
  C[i] = s;
}

size_t gram_smem(int ns) {
  return 1024 + (size_t)GR_STAGES * GR_BR * 4 * 8 * ns + 64 * GR_THREADS * 4 + 2 * GR_STAGES * 8 + 16;
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

// Row splits of the TN reduction: about eight resident waves of CTAs (three
// per SM; short CTAs keep the last wave's tail small), each split at least
// 1024 rows.
int tn_splits(int64_t n, int Ka, int N) {
  const int tiles = (int)(ceil_div(Ka, TN_BT) * ceil_div(N, TN_BT));
  int64_t want = ceil_div(8LL * 3 * sm_count(), tiles);
  const int64_t maxs = std::max<int64_t>(1, ceil_div(n, 1024));
  if (want > maxs) want = maxs;
  if (want > 1024) want = 1024;
  return (int)std::max<int64_t>(1, want);
}

size_t tn_partial_doubles(int64_t n, int Ka, int N) {
  size_t d = (size_t)tn_splits(n, Ka, N) * Ka * N;
  if (Ka == N && Ka <= 8 * GR_MAXNS) d = std::max(d, (size_t)sm_count() * Ka * Ka);   // k_gram_f32's partials
  return d;
}

dmd_status f32_gemm_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const float* B32,
                       float* C, int64_t ldc, cudaStream_t st, const int32_t* skip) {
  if (n <= 0 || N <= 0) return DMD_OK;
  const int ntn = (int)ceil_div(N, NN_BN);
  const int64_t blocks = ceil_div(n, NN_BM) * ntn;
  k_gemm_nn_f32<<<(unsigned)blocks, 256, 0, st>>>(n, Kd, N, A, lda, B32, C, ldc, ntn, skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status f32_gemm_tn(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B,
                       int64_t ldb, double* C, double* part, cudaStream_t st, const int32_t* skip) {
  if (Ka <= 0 || N <= 0) return DMD_OK;
  if (n <= 0 && skip == nullptr) {
    DMD_CUDA_TRY(cudaMemsetAsync(C, 0, (size_t)Ka * N * sizeof(double), st));
    return DMD_OK;
  }
  if (A == B && Ka == N && lda == ldb && Ka <= 8 * GR_MAXNS) {
    // a symmetric Gram: every CTA forms the whole triangle of its row chunk
    const int ns = (int)ceil_div(Ka, 8);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(), ceil_div(n, 1024)));
    const int64_t chunk = round_up(ceil_div(n, grid), GR_BR);
    const int parts = (int)ceil_div(n, chunk);   // every CTA owns rows
    CUtensorMap mA;
    DMD_TRY(make_map(&mA, A, n, Ka, lda, GR_BR, 8 * ns, true));
    const size_t smem = gram_smem(ns);
    DMD_CUDA_TRY(cudaFuncSetAttribute(k_gram_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gram_f32<<<(unsigned)parts, GR_THREADS, smem, st>>>(mA, n, Ka, ns, part, chunk, status_word(), skip);
    DMD_LAUNCH_CHECK();
    const int64_t count = (int64_t)Ka * Ka;
    k_reduce_gram<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(Ka, parts, part, C, skip);
    DMD_LAUNCH_CHECK();
    return DMD_OK;
  }
  int splits = tn_splits(n, Ka, N);
  const int64_t chunk = round_up(ceil_div(n, splits), TN_BR);
  splits = (int)ceil_div(n, chunk);   // every split owns rows
  const int nta = (int)ceil_div(Ka, TN_BT), ntb = (int)ceil_div(N, TN_BT);
  const bool sym = A == B && Ka == N && lda == ldb;
  const int ntiles = sym ? nta * (nta + 1) / 2 : nta * ntb;
  CUtensorMap mA, mB;
  DMD_TRY(make_map(&mA, A, n, Ka, lda, TN_BR, TN_BT, true));
  DMD_TRY(make_map(&mB, B, n, N, ldb, TN_BR, TN_BT, true));
  DMD_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tn_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TN_SMEM));
  k_gemm_tn_f32<<<(unsigned)(ntiles * splits), TN_THREADS, TN_SMEM, st>>>(mA, mB, n, Ka, N, part, nta, ntb, ntiles,
                                                                         sym ? 1 : 0, chunk, status_word(), skip);
  DMD_LAUNCH_CHECK();
  const int64_t count = (int64_t)Ka * N;
  k_reduce_splits<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(Ka, N, splits, part, C, sym ? 1 : 0, skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status f64_to_f32(int64_t count, const double* in, float* out, cudaStream_t st, const int32_t* skip) {
  if (count <= 0) return DMD_OK;
  k_f64_to_f32<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, in, out, skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

int device_sm_count() { return sm_count(); }

}  // namespace dmd
