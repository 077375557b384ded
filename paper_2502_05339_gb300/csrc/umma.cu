// BF16x3 tensor-core passes over the tall snapshot matrices (tcgen05, sm_103a).
//
// Every FP32 operand x is split into bf16 hi = rn(x), lo = rn(x - hi) and a
// product is formed as hi*hi' + hi*lo' + lo*hi' with FP32 accumulation in
// tensor memory (TMEM).  FP32 tiles arrive by TMA (cp.async.bulk.tensor) into a
// shared-memory ring; converter warps split them into the K-major canonical
// UMMA layout (no swizzle: 8-row x 16-byte core matrices, K-adjacent core
// matrices 128 B apart, 8-row groups 256 B apart); one thread issues the
// tcgen05.mma instructions; epilogue warps drain TMEM with tcgen05.ld.
// All waits are bounded (2 s on the global timer); a wait that runs out sets
// an abort flag that every role checks, the kernel finishes its in-flight
// asynchronous work, frees TMEM and reports DMD_ETIMEOUT.
//
//   k_umma_nn_bres : C = A B, A tall (n x Kd) streamed, B (Kd x N, N <= 256)
//                    resident in shared memory -- sketch X Omega, power step
//                    X Z, CholeskyQR step Y R^{-1}, modes X' M (Sec. 4.3, 3.1).
//   k_umma_nn_ares : C = A B with A's 128-row tile resident in TMEM and B streamed in
//                    column chunks -- the reconstruction Phi_R C of
//                    Eq. large_time_step with K frames.
//   k_umma_tn      : C = A^T B reduced over the tall dimension -- X^T Q, Q^T S
//                    and Gram matrices; per-CTA FP64 partials; 2- or 3-way
//                    bf16 split (3 or 6 products).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace dmd {

namespace {

// ---------------------------------------------------- B operand pre-split

// B (Kd x N, FP64, column-major, ld Kd) -> bf16 hi/lo in the UMMA K-slice
// layout of an N-row operand, grouped in column chunks of BN rows:
// chunk c, slice s, row j: offset c*(2*ks*BN*32) + s*BN*32 + chunk-of(j, k); lo
// follows hi inside each chunk (ks*BN*32 bytes later).  Zero padded.
__global__ void k_split_b(int Kd, int N, const double* __restrict__ B, int BN, int ksteps, int nchunks,
                          uint8_t* __restrict__ out, const int32_t* __restrict__ skip = nullptr) {
  if (skip != nullptr && *skip != 0) return;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // one thread per (row, slice)
  const int64_t total = (int64_t)nchunks * BN * ksteps;
  if (idx >= total) return;
  const int jr = (int)(idx % BN);
  const int s = (int)((idx / BN) % ksteps);
  const int c = (int)(idx / ((int64_t)BN * ksteps));
  const int j = c * BN + jr;
  float x[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int k = s * 16 + t;
    x[t] = (j < N && k < Kd) ? (float)B[(int64_t)j * Kd + k] : 0.f;
  }
  uint8_t* base = out + (int64_t)c * (2LL * ksteps * BN * 32);
  uint8_t* hi = base + (int64_t)s * BN * 32;
  uint8_t* lo = base + (int64_t)(ksteps + s) * BN * 32;
  // residual of the FP64 value: use x (FP32) for hi, the FP64 remainder for lo
  uint32_t h[8], l[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float v0 = x[2 * i], v1 = x[2 * i + 1];
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
    double r0 = 0.0, r1 = 0.0;
    const int k0 = s * 16 + 2 * i;
    if (j < N && k0 < Kd) r0 = B[(int64_t)j * Kd + k0] - (double)__bfloat162float(h0);
    if (j < N && k0 + 1 < Kd) r1 = B[(int64_t)j * Kd + k0 + 1] - (double)__bfloat162float(h1);
    h[i] = pack2(h0, h1);
    l[i] = pack2(__float2bfloat16_rn((float)r0), __float2bfloat16_rn((float)r1));
  }
  *reinterpret_cast<uint4*>(hi + kslice_off(jr, 0)) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(hi + kslice_off(jr, 1)) = make_uint4(h[4], h[5], h[6], h[7]);
  *reinterpret_cast<uint4*>(lo + kslice_off(jr, 0)) = make_uint4(l[0], l[1], l[2], l[3]);
  *reinterpret_cast<uint4*>(lo + kslice_off(jr, 1)) = make_uint4(l[4], l[5], l[6], l[7]);
}

// ============================================================ NN, B resident

constexpr int NN_SMAX = 12; // TMA stages (FP32 128 x 16 tiles, 8 KB): as many as fit, up to 12
constexpr int NN_CS = 4;   // converted stages (bf16 hi + lo, 8 KB)
constexpr int NN_CONV = 8; // converter warps: two per 32-row group, one per 8-wide half of a K-slice
constexpr int NN_THREADS = 32 * (2 + NN_CONV + 4);

__global__ void __launch_bounds__(NN_THREADS, 1)
    k_umma_nn_bres(const __grid_constant__ CUtensorMap tmA, const uint8_t* __restrict__ Bsplit,
                   float* __restrict__ C, int64_t ldc, int64_t n, int N, int Np, int ksteps, int64_t ntiles,
                   int ns, int32_t* err, const int32_t* __restrict__ skip) {
  // a device-side flag (work that a device decision made unnecessary): every
  // CTA reads the same value before any barrier or tensor-memory allocation
  if (skip != nullptr && *skip != 0) return;
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1024(smraw);
  const uint32_t bres_bytes = 2u * (uint32_t)ksteps * (uint32_t)Np * 32u;
  uint8_t* Bres = sm;
  uint8_t* stA = sm + ((bres_bytes + 1023u) & ~1023u);
  uint8_t* cv = stA + ns * 8192;
  uint64_t* bars = reinterpret_cast<uint64_t*>(cv + NN_CS * 8192);
  uint64_t* full = bars;
  uint64_t* empty = full + NN_SMAX;
  uint64_t* cfull = empty + NN_SMAX;
  uint64_t* cempty = cfull + NN_CS;
  uint64_t* accf = cempty + NN_CS;
  uint64_t* acce = accf + 2;
  uint64_t* bfull = acce + 2;
  uint64_t* tdown = bfull + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tdown + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < ns; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 32 * NN_CONV);
    }
    for (int i = 0; i < NN_CS; ++i) {
      mbar_init(&cfull[i], 32 * NN_CONV);
      mbar_init(&cempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 128);
    }
    mbar_init(bfull, 1);
    mbar_init(tdown, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tslot, 512);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      mbar_expect_tx(bfull, bres_bytes);
      for (uint32_t off = 0; off < bres_bytes; off += 32768u)
        bulk_g2s(Bres + off, Bsplit + off, min(32768u, bres_bytes - off), bfull);
      uint32_t it = 0;
      uint32_t last_par[NN_SMAX];
      bool issued[NN_SMAX];
      for (int i = 0; i < NN_SMAX; ++i) issued[i] = false, last_par[i] = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        for (int ks = 0; ks < ksteps; ++ks, ++it) {
          const uint32_t s = it % ns;
          if (!mbar_wait(&empty[s], ((it / ns) & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], 8192);
          tma_load_2d(stA + s * 8192, &tmA, &full[s], (int)(tile * 128), ks * 16);
          issued[s] = true;
          last_par[s] = (it / ns) & 1;
        }
      }
      // in-flight TMA writes must land before the CTA's shared memory goes away
      for (int i = 0; i < ns; ++i)
        if (issued[i]) mbar_wait_drain(&full[i], last_par[i]);
      mbar_wait_drain(bfull, 0);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, Np);
      const uint64_t a0d = sdesc(su32(cv), kLBO, kSBO), b0d = sdesc(su32(Bres), kLBO, kSBO);
      const uint32_t b_step = ((uint32_t)Np * 32u) >> 4, b_lo = ((uint32_t)ksteps * (uint32_t)Np * 32u) >> 4;
      bool ok = mbar_wait(bfull, 0, abort_flag);
      uint32_t cit = 0, ait = 0;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++ait) {
        const uint32_t ab = ait & 1;
        if (!mbar_wait(&acce[ab], ((ait >> 1) & 1) ^ 1, abort_flag)) break;
        tc_after();
        const uint32_t d = tmem + ab * 256;
        for (int ks = 0; ks < ksteps; ++ks, ++cit) {
          const uint32_t cs = cit % NN_CS;
          if (!mbar_wait(&cfull[cs], (cit / NN_CS) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_after();
          // descriptors by offset from precomputed bases (16-byte units)
          const uint64_t ahd = a0d + (uint64_t)(cs * 512u), ald = ahd + 256u;
          const uint64_t bhd = b0d + (uint64_t)((uint32_t)ks * b_step), bld = bhd + b_lo;
          umma_bf16(d, ahd, bhd, idesc, ks > 0 ? 1u : 0u);
          umma_bf16(d, ahd, bld, idesc, 1u);
          umma_bf16(d, ald, bhd, idesc, 1u);
          umma_commit(&cempty[cs]);
        }
        if (!ok) break;
        umma_commit(&accf[ab]);
      }
      umma_commit(tdown);          // completes when every MMA issued above has finished
      mbar_wait_drain(tdown, 0);
    }
  } else if (warp < 2 + NN_CONV) {
    // converters: thread t splits row t % 128 of the tile, K-columns
    // 8 h .. 8 h + 7 of each slice (h = t / 128: one 16-byte chunk per plane)
    const int t = threadIdx.x - 64;
    const int row = t & 127, h = t >> 7;
    uint32_t it = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      for (int ks = 0; ks < ksteps; ++ks, ++it) {
        const uint32_t s = it % ns, cs = it % NN_CS;
        if (!mbar_wait(&full[s], (it / ns) & 1, abort_flag) ||
            !mbar_wait(&cempty[cs], ((it / NN_CS) & 1) ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        const float* src = reinterpret_cast<const float*>(stA + s * 8192) + 8 * h * 128 + row;
        uint32_t hv[4], lv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float x0 = src[(2 * i) * 128], x1 = src[(2 * i + 1) * 128];
          const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
          hv[i] = pack2(h0, h1);
          lv[i] = pack2(__float2bfloat16_rn(x0 - __bfloat162float(h0)), __float2bfloat16_rn(x1 - __bfloat162float(h1)));
        }
        uint8_t* dst = cv + cs * 8192 + kslice_off(row, h);
        *reinterpret_cast<uint4*>(dst) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<uint4*>(dst + 4096) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
        fence_async_smem();
        mbar_arrive(&cfull[cs]);
        mbar_arrive(&empty[s]);
      }
    }
  } else {
    const int q = warp & 3;
    const int rowq = q * 32 + lane;
    uint32_t ait = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++ait) {
      const uint32_t ab = ait & 1;
      if (!mbar_wait(&accf[ab], (ait >> 1) & 1, abort_flag)) break;
      tc_after();
      const int64_t row = tile * 128 + rowq;
      for (int c0 = 0; c0 < Np; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ab * 256 + (uint32_t)c0 + ((uint32_t)(q * 32) << 16), v);
        if (row < n) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < N) C[(int64_t)(c0 + j) * ldc + row] = v[j];
        }
      }
      tc_before();
      mbar_arrive(&acce[ab]);
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    tc_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(abort_flag)) raise_status(err, DMD_ETIMEOUT, 8001);
}

// ============================================================ NN, A resident

constexpr int AR_MAXSA = 4;  // TMA stages for the A tile slices (runtime sa <= 4)
constexpr int AR_MAXNB = 4;  // B ring entries (runtime nb <= 4)
constexpr int AR_MAXKS = 16; // K-slices of the resident A tile (Kd <= 256)
constexpr int AR_ACC = 2;    // TMEM accumulators (bn columns each)
constexpr int AR_THREADS = 448;           // producer, issuer, 4 converters, 2 x 4 epilogue warps
constexpr uint32_t AR_STG = 8 * 2 * 2048;   // epilogue staging: 8 warps x 2 buffers x 2 KB

// Widest frame chunk (a multiple of 16, at most 256) whose two accumulators
// fit beside the resident A tile (16 columns per K-slice: hi, then lo) in the
// 512 tensor-memory columns: 176 frames at 150 modes.
constexpr int ares_bn_max(int ksteps) {
  return ((512 - 16 * ksteps) / 2 / 16 * 16) < 256 ? ((512 - 16 * ksteps) / 2 / 16 * 16) : 256;
}

// C = A B with the 128-row tile of A resident in TENSOR memory (split into
// bf16 hi / lo by the converter warps and written with tcgen05.st: lane =
// row, 8 columns per 16-wide K-slice), the coefficient matrix B streamed in
// bn-column chunks through a shared-memory ring whose entries hold G K-slices
// of a chunk (hi and lo planes).  A tcgen05.mma holds its issuer for ~100-160
// cycles whatever N (measured), so the chunk is as wide as tensor memory
// allows: two bn-column accumulators beside A, M = 128, N = bn.
// Two sets of four epilogue warps drain the two accumulators (set h takes the
// chunks in accumulator h), so each set has two chunks' product time for one
// chunk's epilogue; each warp writes its 32 rows in 16-column TMA stores
// through a double-buffered 2 KB staging area.
//
// kLoss != 0: the frames are not stored.  The epilogue forms each frame's
// residual against the target field, e = x - tgt (row-wise), and accumulates
// the weighted per-frame loss w_j rho(e) of the streamed objective: rho(e) =
// e^2 / 2, or with delta > 0 the Huber function (e^2 / 2 for |e| <= delta,
// delta (|e| - delta / 2) beyond).  Each thread sums one chunk of its row in
// FP32 and carries the chunk sums in FP64; the CTA's sum (fixed order) goes
// to loss_part[blockIdx.x].  Phi_R is read once per call.
template <int kLoss>
__global__ void __launch_bounds__(AR_THREADS, 1)
    k_umma_nn_ares(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmC,
                   const uint8_t* __restrict__ Bchunks, int64_t n, int N, int ksteps, int bn, int sa, int nb, int G,
                   int nchunks, int64_t ntiles, const float* __restrict__ tgt, const double* __restrict__ wgt,
                   float delta, double* __restrict__ loss_part, int32_t* err, const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;   // as in k_umma_nn_bres
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1024(smraw);
  const uint32_t slice_bytes = (uint32_t)bn * 32u;   // one K-slice of one plane of a chunk
  const uint32_t chunk_bytes = 2u * (uint32_t)ksteps * slice_bytes;
  const uint32_t estride = (2u * (uint32_t)G * slice_bytes + 1023u) & ~1023u;
  const int nent = (ksteps + G - 1) / G;   // ring entries per chunk
  uint8_t* stA = sm;
  uint8_t* Bbuf = stA + sa * 8192;
  uint8_t* stg = Bbuf + nb * estride;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + AR_STG);
  uint64_t* afull = bars;               // TMA slice landed
  uint64_t* aempty = afull + AR_MAXSA;  // slice converted
  uint64_t* bfull = aempty + AR_MAXSA;
  uint64_t* bempty = bfull + AR_MAXNB;
  uint64_t* accf = bempty + AR_MAXNB;
  uint64_t* acce = accf + AR_ACC;
  uint64_t* ares_full = acce + AR_ACC;  // [AR_MAXKS]: slice ks of the tile's A is in TMEM
  uint64_t* ares_free = ares_full + AR_MAXKS;  // MMAs of the tile finished reading A
  uint64_t* tdown = ares_free + 1;
  double* red = reinterpret_cast<double*>(tdown + 1);   // 8 epilogue warps' loss sums
  uint32_t* tslot = reinterpret_cast<uint32_t*>(red + 8);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < AR_MAXSA; ++i) {
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 128);
    }
    for (int i = 0; i < AR_MAXNB; ++i) {
      mbar_init(&bfull[i], 1);
      mbar_init(&bempty[i], 1);
    }
    for (int i = 0; i < AR_ACC; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 128);
    }
    for (int i = 0; i < AR_MAXKS; ++i) mbar_init(&ares_full[i], 128);
    mbar_init(ares_free, 1);
    mbar_init(tdown, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tslot, 512);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;
  const uint32_t acol = (uint32_t)(AR_ACC * bn);   // resident A: hi from here, lo 8 ks columns on

  if (warp == 0) {
    if (lane == 0) {
      uint32_t ait = 0, bit = 0;
      bool ok = true;
      bool a_issued[AR_MAXSA] = {false, false, false, false}, b_issued[AR_MAXNB] = {false, false, false, false};
      uint32_t a_par[AR_MAXSA] = {0, 0, 0, 0}, b_par[AR_MAXNB] = {0, 0, 0, 0};
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        for (int ks = 0; ks < ksteps; ++ks, ++ait) {
          const uint32_t s = ait % sa;
          if (!mbar_wait(&aempty[s], ((ait / sa) & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&afull[s], 8192);
          tma_load_2d(stA + s * 8192, &tmA, &afull[s], (int)(tile * 128), ks * 16);
          a_issued[s] = true;
          a_par[s] = (ait / sa) & 1;
        }
        for (int c = 0; ok && c < nchunks; ++c) {
          const uint8_t* src = Bchunks + (int64_t)c * chunk_bytes;
          for (int e = 0; e < nent; ++e, ++bit) {
            const uint32_t b = bit % nb;
            if (!mbar_wait(&bempty[b], ((bit / nb) & 1) ^ 1, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t s0 = (uint32_t)(e * G), gs = (uint32_t)min(G, ksteps - e * G);
            const uint32_t bytes = gs * slice_bytes;
            mbar_expect_tx(&bfull[b], 2u * bytes);
            uint8_t* dst = Bbuf + b * estride;
            for (uint32_t off = 0; off < bytes; off += 32768u) {
              const uint32_t len = min(32768u, bytes - off);
              bulk_g2s(dst + off, src + s0 * slice_bytes + off, len, &bfull[b]);
              bulk_g2s(dst + (uint32_t)G * slice_bytes + off, src + ((uint32_t)ksteps + s0) * slice_bytes + off, len,
                       &bfull[b]);
            }
            b_issued[b] = true;
            b_par[b] = (bit / nb) & 1;
          }
        }
      }
      for (int i = 0; i < sa; ++i)
        if (a_issued[i]) mbar_wait_drain(&afull[i], a_par[i]);
      for (int i = 0; i < nb; ++i)
        if (b_issued[i]) mbar_wait_drain(&bfull[i], b_par[i]);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, bn);
      const uint32_t a_hi = tmem + acol, a_lo = tmem + acol + (uint32_t)ksteps * 8u;
      // descriptors advance by offsets (address field in 16-byte units)
      const uint64_t bstep = (uint64_t)(slice_bytes >> 4), blo = (uint64_t)(((uint32_t)G * slice_bytes) >> 4);
      uint32_t tit = 0, bit = 0, accit = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tit) {
        for (int c = 0; ok && c < nchunks; ++c, ++accit) {
          const uint32_t ab = accit % AR_ACC;
          if (!mbar_wait(&acce[ab], ((accit / AR_ACC) & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_after();
          const uint32_t d = tmem + ab * (uint32_t)bn;
          for (int e = 0; e < nent; ++e, ++bit) {
            const uint32_t b = bit % nb;
            if (!mbar_wait(&bfull[b], (bit / nb) & 1, abort_flag)) {
              ok = false;
              break;
            }
            tc_after();
            const int s0 = e * G, gs = min(G, ksteps - e * G);
            uint64_t bhd = sdesc(su32(Bbuf + b * estride), kLBO, kSBO);
            uint32_t ah = a_hi + (uint32_t)s0 * 8u, al = a_lo + (uint32_t)s0 * 8u;
            if (c == 0) {   // the tile's first chunk follows the conversion slice by slice
              for (int s = 0; s < gs; ++s, bhd += bstep, ah += 8u, al += 8u) {
                if (!mbar_wait(&ares_full[s0 + s], tit & 1, abort_flag)) {
                  ok = false;
                  break;
                }
                tc_after();
                umma_bf16_ta(d, ah, bhd, idesc, (s0 + s) > 0 ? 1u : 0u);
                umma_bf16_ta(d, ah, bhd + blo, idesc, 1u);
                umma_bf16_ta(d, al, bhd, idesc, 1u);
              }
              if (!ok) break;
            } else {
              // the issue loop holds nothing but the products and the
              // descriptor offsets (every extra instruction slows the issue)
              const uint64_t bend = bhd + (uint64_t)gs * bstep;
              if (s0 == 0) {
                umma_bf16_ta(d, ah, bhd, idesc, 0u);
                umma_bf16_ta(d, ah, bhd + blo, idesc, 1u);
                umma_bf16_ta(d, al, bhd, idesc, 1u);
                bhd += bstep;
                ah += 8u;
                al += 8u;
              }
              for (; bhd < bend; bhd += bstep, ah += 8u, al += 8u) {
                umma_bf16_ta(d, ah, bhd, idesc, 1u);
                umma_bf16_ta(d, ah, bhd + blo, idesc, 1u);
                umma_bf16_ta(d, al, bhd, idesc, 1u);
              }
            }
            umma_commit(&bempty[b]);
          }
          if (!ok) break;
          umma_commit(&accf[ab]);
        }
        if (!ok) break;
        umma_commit(ares_free);
      }
      umma_commit(tdown);
      mbar_wait_drain(tdown, 0);
    }
  } else if (warp < 6) {
    // converters: warp w owns TMEM lanes 32 (w % 4) .. + 31, i.e. those rows of the tile
    const int q = warp & 3;
    const int t = q * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    uint32_t ait = 0, tit = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tit) {
      // the previous tile's MMAs must be done with the resident A
      if (tit > 0 && !mbar_wait(ares_free, (tit - 1) & 1, abort_flag)) break;
      tc_after();
      for (int ks = 0; ks < ksteps; ++ks, ++ait) {
        const uint32_t s = ait % sa;
        if (!mbar_wait(&afull[s], (ait / sa) & 1, abort_flag)) {
          ok = false;
          break;
        }
        const float* src = reinterpret_cast<const float*>(stA + s * 8192);
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float x0 = src[(2 * i) * 128 + t], x1 = src[(2 * i + 1) * 128 + t];
          const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
          h[i] = pack2(h0, h1);
          l[i] = pack2(__float2bfloat16_rn(x0 - __bfloat162float(h0)), __float2bfloat16_rn(x1 - __bfloat162float(h1)));
        }
        tmem_st8(tmem + acol + (uint32_t)ks * 8u + lane_base, h);
        tmem_st8(tmem + acol + (uint32_t)(ksteps + ks) * 8u + lane_base, l);
        tmem_st_wait();
        mbar_arrive(&aempty[s]);
        tc_before();
        mbar_arrive(&ares_full[ks]);
      }
      if (!ok) break;
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; set h = the accumulator it drains
    const int q = warp & 3, ew = warp - 6, h = ew >> 2;
    float* mystg = reinterpret_cast<float*>(stg + (uint32_t)ew * 2u * 2048u);
    uint32_t accit = 0;
    int sbuf = 0;
    bool ok = true;
    double lacc = 0.0;   // kLoss: this thread's (row's) loss
    // kLoss: every frame's weight as FP32, zero past N, in the staging area
    // (whole chunks; the loss launcher keeps nchunks * bn <= 4096)
    float* wall = reinterpret_cast<float*>(stg);
    if (kLoss) {
      for (int j = threadIdx.x - 192; j < nchunks * bn; j += 256) wall[j] = j < N ? (float)wgt[j] : 0.f;
      asm volatile("bar.sync 1, 256;" ::: "memory");   // the eight epilogue warps
    }
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      const int row0 = (int)(tile * 128) + q * 32;
      const bool row_ok = (int64_t)row0 + lane < n;
      const float tv = (kLoss && row_ok) ? tgt[row0 + lane] : 0.f;
      for (int c = 0; c < nchunks; ++c, ++accit) {
        const uint32_t ab = accit % AR_ACC;
        if ((int)ab != h) continue;
        if (!mbar_wait(&accf[ab], (accit / AR_ACC) & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_after();
        const int cend = min(bn, N - c * bn);   // the last chunk may be ragged
        const uint32_t acc = tmem + ab * (uint32_t)bn + ((uint32_t)(q * 32) << 16);
        if (kLoss) {
          // up to 64 columns per round: the round's loads in flight, one
          // wait; columns past the chunk's frames are selected away (their
          // accumulator entries may hold anything)
          const float* wc = wall + c * bn;
          float s = 0.f;
          for (int c0 = 0; c0 < cend; c0 += 64) {
            uint32_t v[64];
            const int rem = cend - c0;   // the same in every lane
            tmem_ld16_nw(acc + (uint32_t)c0, v);
            if (rem > 16) tmem_ld16_nw(acc + (uint32_t)c0 + 16u, v + 16);
            if (rem > 32) tmem_ld16_nw(acc + (uint32_t)c0 + 32u, v + 32);
            if (rem > 48) tmem_ld16_nw(acc + (uint32_t)c0 + 48u, v + 48);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 64; ++j) {
              const bool in = j < rem;
              const float wj = wc[c0 + (in ? j : 0)];
              const float e = __uint_as_float(v[j]) - tv, ae = fabsf(e);
              const float rho = (delta > 0.f && ae > delta) ? delta * (ae - 0.5f * delta) : 0.5f * e * e;
              s += in ? wj * rho : 0.f;
            }
          }
          if (row_ok) lacc += (double)s;
          tc_before();
          mbar_arrive(&acce[ab]);
          continue;
        }
        for (int c0 = 0; c0 < cend; c0 += 16) {
          float v[16];
          tmem_ld16(acc + (uint32_t)c0, v);
          // the store issued two rounds ago from this buffer must have read it
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          __syncwarp();
          float* buf = mystg + sbuf * 512;
#pragma unroll
          for (int j = 0; j < 16; ++j) buf[j * 32 + lane] = v[j];
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tmC, buf, row0, c * bn + c0);
            bulk_commit();
          }
          sbuf ^= 1;
        }
        tc_before();
        mbar_arrive(&acce[ab]);
      }
    }
    if (kLoss) {
      const double ws = warp_sum(lacc);
      if (lane == 0) red[ew] = ws;
    } else if (lane == 0) {
      bulk_wait0();
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    tc_after();
    tmem_dealloc(tmem, 512);
  }
  if (kLoss && threadIdx.x == 0)
    loss_part[blockIdx.x] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(abort_flag)) raise_status(err, DMD_ETIMEOUT, 8002);
}

// ============================================================ TN reduction

constexpr int TN_S = 4;            // TMA stages (A slice + B slice)
constexpr int TN_CONV = 16;        // converter warps
constexpr int TN_THREADS = 32 * (2 + TN_CONV + 4);

// Split 4 consecutive-K FP32 values of operand row `row` (K offset 4*qd in
// the 16-wide slice) into NS bf16 planes `plane` bytes apart (hi, then the
// rounded remainders).
template <int NS>
__device__ __forceinline__ void split_store4(float4 v, uint8_t* base, uint32_t plane, int row, int qd) {
  const uint32_t off = kslice_off(row, qd >> 1) + (uint32_t)(qd & 1) * 8u;
  const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
  const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
  const float r0 = v.x - f01.x, r1 = v.y - f01.y, r2 = v.z - f23.x, r3 = v.w - f23.y;
  const __nv_bfloat162 m01 = __floats2bfloat162_rn(r0, r1), m23 = __floats2bfloat162_rn(r2, r3);
  *reinterpret_cast<uint2*>(base + off) = make_uint2(bf2_bits(h01), bf2_bits(h23));
  *reinterpret_cast<uint2*>(base + plane + off) = make_uint2(bf2_bits(m01), bf2_bits(m23));
  if (NS == 3) {
    const float2 g01 = __bfloat1622float2(m01), g23 = __bfloat1622float2(m23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(r0 - g01.x, r1 - g01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(r2 - g23.x, r3 - g23.y);
    *reinterpret_cast<uint2*>(base + 2 * plane + off) = make_uint2(bf2_bits(l01), bf2_bits(l23));
  }
}

// Converter loop over one k-step (half h of a 32-row stage): unit u is
// operand row u / 4 (a column of the box: one 128-byte line, 16-byte chunks
// XOR-swizzled by the line index mod 8), K offset 4 * (u % 4), read from
// chunk 4 h + u % 4 of that line; written into NS planes.
template <int NS>
__device__ __forceinline__ void split_slice(const float4* src, int units, int h, uint8_t* base, uint32_t plane, int t,
                                            int nthreads) {
#pragma unroll 4
  for (int u = t; u < units; u += nthreads) {
    const int col = u >> 2, q = u & 3;
    const float4 v = src[col * 8 + ((h * 4 + q) ^ (col & 7))];
    split_store4<NS>(v, base, plane, col, q);
  }
}

// part[blockIdx.x][b * Ka + a] = sum over this CTA's rows of A[:, a] * B[:, b].
// A slice: TMA box {16 rows, Mt*128 cols}; B slice: box {16 rows, Np cols}.
// nsplit = 2: bf16 hi + lo, products hh + hl + lh (BF16x3).  nsplit = 3:
// hi + mid + lo, products hh + hm + mh + hl + lh + mm.  sym != 0: B is A
// (a Gram matrix), loaded and split once.  Roles: warp 0 TMA producer, warp 1
// MMA issuer, TN_CONV converter warps (FP32 slice -> bf16 planes; each warp
// reads 512 contiguous bytes per step, four lanes per operand row), four
// epilogue warps (TMEM -> FP64 partial every `flush` k-steps).
__global__ void __launch_bounds__(TN_THREADS, 1)
    k_umma_tn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n, int Ka,
              int N, int Mt, int Np, int nsplit, int flush, int sym, int ns, int64_t chunk,
              double* __restrict__ part, int32_t* err, const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;   // as in k_umma_nn_bres
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1024(smraw);
  // a TMA stage holds 32 rows of n (two k-steps): 128 contiguous bytes per
  // column, laid out with the 128-byte swizzle
  const uint32_t a_bytes = 32u * 4u * (uint32_t)Mt * 128u;        // FP32 rows of A
  const uint32_t b_bytes = sym ? 0u : 32u * 4u * (uint32_t)Np;   // FP32 rows of B
  const uint32_t st_bytes = (32u * 4u * (uint32_t)Mt * 128u + 32u * 4u * (uint32_t)Np + 1023u) & ~1023u;
  const uint32_t ca_bytes = (uint32_t)Mt * 128u * 32u;       // one bf16 K-slice plane of A
  const uint32_t cb_bytes = (uint32_t)Np * 32u;
  const uint32_t cv_bytes = ((uint32_t)nsplit * (ca_bytes + cb_bytes) + 1023u) & ~1023u;
  uint8_t* st = sm;
  uint8_t* cv = st + ns * st_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(cv + 2 * cv_bytes);
  uint64_t* full = bars;
  uint64_t* empty = full + TN_S;
  uint64_t* cfull = empty + TN_S;      // 2 converted buffers
  uint64_t* cempty = cfull + 2;
  uint64_t* accf = cempty + 2;
  uint64_t* acce = accf + 1;
  uint64_t* tdown = acce + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tdown + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t rbeg = (int64_t)blockIdx.x * chunk;
  const int64_t rend = min(n, rbeg + chunk);
  // k-steps of 16 rows, rounded up to whole stages (rows past this CTA's
  // range are past n: chunk is a multiple of 32, and TMA fills zeros there)
  const int ksteps = rend > rbeg ? 2 * (int)((rend - rbeg + 31) / 32) : 0;
  const int nstage = ksteps / 2;
  const int nflush = (ksteps + flush - 1) / flush;
  constexpr int kConvThreads = 32 * TN_CONV;

  if (threadIdx.x == 0) {
    for (int i = 0; i < ns; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConvThreads);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&cfull[i], kConvThreads);
      mbar_init(&cempty[i], 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 128);
    mbar_init(tdown, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tslot, 512);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      bool issued[TN_S] = {false, false, false, false};
      uint32_t par[TN_S] = {0, 0, 0, 0};
      for (int g = 0; g < nstage; ++g) {
        const uint32_t s = g % ns;
        if (!mbar_wait(&empty[s], ((g / ns) & 1) ^ 1, abort_flag)) break;
        mbar_expect_tx(&full[s], a_bytes + b_bytes);
        const int r0 = (int)(rbeg + (int64_t)g * 32);
        tma_load_2d(st + s * st_bytes, &tmA, &full[s], r0, 0);
        if (!sym) tma_load_2d(st + s * st_bytes + a_bytes, &tmB, &full[s], r0, 0);
        issued[s] = true;
        par[s] = (g / ns) & 1;
      }
      for (int i = 0; i < ns; ++i)
        if (issued[i]) mbar_wait_drain(&full[i], par[i]);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(128, Np);
      const uint64_t dbase = sdesc(su32(cv), kLBO, kSBO);
      const uint32_t cv_off = cv_bytes >> 4, a_plane = ca_bytes >> 4;
      const uint32_t b_off = sym ? 0u : ((uint32_t)nsplit * ca_bytes) >> 4;
      const uint32_t b_plane = (sym ? ca_bytes : cb_bytes) >> 4;
      bool ok = true;
      int ks = 0;
      for (int f = 0; ok && f < nflush; ++f) {
        if (!mbar_wait(acce, (f & 1) ^ 1, abort_flag)) break;
        tc_after();
        const int kend = min(ksteps, (f + 1) * flush);
        for (int kk = 0; ks < kend; ++ks, ++kk) {
          const uint32_t cs = ks & 1;
          if (!mbar_wait(&cfull[cs], (ks >> 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_after();
          // descriptors by offset from the first buffer's (address field in
          // 16-byte units, far from overflowing): B planes follow the A
          // planes; a Gram reads A's planes twice
          const uint64_t base = dbase + (uint64_t)(cs * cv_off);
          const uint64_t b0 = base + b_off, b1 = b0 + b_plane, b2 = b1 + b_plane;
          const uint32_t acc = kk > 0 ? 1u : 0u;
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            if (mt >= Mt) break;
            const uint32_t d = tmem + (uint32_t)(mt * Np);
            const uint64_t a0 = base + (uint64_t)(mt * 256), a1 = a0 + a_plane, a2 = a1 + a_plane;
            umma_bf16(d, a0, b0, idesc, acc);
            umma_bf16(d, a0, b1, idesc, 1u);
            umma_bf16(d, a1, b0, idesc, 1u);
            if (nsplit == 3) {
              umma_bf16(d, a0, b2, idesc, 1u);
              umma_bf16(d, a2, b0, idesc, 1u);
              umma_bf16(d, a1, b1, idesc, 1u);
            }
          }
          umma_commit(&cempty[cs]);
        }
        if (!ok) break;
        umma_commit(accf);
      }
      umma_commit(tdown);
      mbar_wait_drain(tdown, 0);
    }
  } else if (warp < 2 + TN_CONV) {
    const int t = threadIdx.x - 64;
    // float4 units per k-step: valid operand rows only.  The padding rows of
    // the converted planes (A rows Ka .. Mt*128, B rows N .. Np) are zeroed
    // once here and never written again.
    const int na4 = Ka * 4, nb4 = sym ? 0 : N * 4;
    {
      const int pa = Mt * 128 - Ka, pb = sym ? 0 : Np - N;
      const int per_plane = 2 * (pa + pb);   // 16-byte chunks: 2 per row
      const int total = 2 * nsplit * per_plane;
      for (int i = t; i < total; i += kConvThreads) {
        const int buf = i / (nsplit * per_plane);
        const int rem = i % (nsplit * per_plane);
        const int plane = rem / per_plane;
        const int c = rem % per_plane;
        const int row = c >> 1, half = c & 1;
        uint8_t* base = cv + buf * cv_bytes;
        uint8_t* dst = row < pa ? base + plane * ca_bytes + kslice_off(Ka + row, half)
                                : base + nsplit * ca_bytes + plane * cb_bytes + kslice_off(N + row - pa, half);
        *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    for (int ks = 0; ks < ksteps; ++ks) {
      const int g = ks >> 1, h = ks & 1;
      const uint32_t s = g % ns, cs = ks & 1;
      if ((h == 0 && !mbar_wait(&full[s], (g / ns) & 1, abort_flag)) ||
          !mbar_wait(&cempty[cs], ((ks >> 1) & 1) ^ 1, abort_flag))
        break;
      const float4* sa = reinterpret_cast<const float4*>(st + s * st_bytes);
      const float4* sb = reinterpret_cast<const float4*>(st + s * st_bytes + a_bytes);
      uint8_t* base = cv + cs * cv_bytes;
      uint8_t* bb = base + (uint32_t)nsplit * ca_bytes;
      if (nsplit == 3) {
        split_slice<3>(sa, na4, h, base, ca_bytes, t, kConvThreads);
        split_slice<3>(sb, nb4, h, bb, cb_bytes, t, kConvThreads);
      } else {
        split_slice<2>(sa, na4, h, base, ca_bytes, t, kConvThreads);
        split_slice<2>(sb, nb4, h, bb, cb_bytes, t, kConvThreads);
      }
      fence_async_smem();
      mbar_arrive(&cfull[cs]);
      if (h == 1) mbar_arrive(&empty[s]);
    }
  } else {
    const int q = warp & 3;
    const int rowq = q * 32 + lane;
    double* out = part + (int64_t)blockIdx.x * Ka * N;
    for (int f = 0; f < nflush; ++f) {
      if (!mbar_wait(accf, f & 1, abort_flag)) break;
      tc_after();
      for (int mt = 0; mt < Mt; ++mt) {
        const int a = mt * 128 + rowq;
        for (int c0 = 0; c0 < Np; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + (uint32_t)(mt * Np + c0) + ((uint32_t)(q * 32) << 16), v);
          // Each partial entry has one owner thread, so its additions land in
          // program order (deterministic); a reduction needs no round trip.
          if (a < Ka) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int b = c0 + j;
              if (b < N) {
                double* p = out + (int64_t)b * Ka + a;
                if (f == 0) *p = (double)v[j];
                else atomicAdd(p, (double)v[j]);
              }
            }
          }
        }
      }
      tc_before();
      mbar_arrive(acce);
    }
    if (nflush == 0) {   // no rows for this CTA: its partial is zero
      for (int mt = 0; mt < Mt; ++mt) {
        const int a = mt * 128 + rowq;
        if (a < Ka)
          for (int b = 0; b < N; ++b) out[(int64_t)b * Ka + a] = 0.0;
      }
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    tc_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(abort_flag)) raise_status(err, DMD_ETIMEOUT, 8003);
}

// C[a0 + a, b0 + b] (ld ldc) = sum over the CTAs' partials (ka x nb each), fixed order.
// With trans != 0 the block is written transposed: C[a, b] goes to C[b + a * ldc].
__global__ void k_reduce_parts(int ka, int nb, int parts, const double* __restrict__ part, double* __restrict__ C,
                               int64_t ldc, int trans, const int32_t* __restrict__ skip) {
  if (skip != nullptr && *skip != 0) return;
  const int64_t count = (int64_t)ka * nb;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += part[(int64_t)p * count + i];
  const int a = (int)(i % ka), b = (int)(i / ka);
  if (trans) C[(int64_t)a * ldc + b] = s;
  else C[(int64_t)b * ldc + a] = s;
}

// ------------------------------------------------------------ host side

}  // namespace

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  return sms;
}

namespace {

constexpr int kMaxSmem = 227 * 1024;

size_t bres_smem(int ksteps, int Np, int ns) {
  return 1024 + (((size_t)2 * ksteps * Np * 32 + 1023) & ~(size_t)1023) + (size_t)ns * 8192 + NN_CS * 8192 + 512;
}
// TMA stages of the B-resident kernel: as many as fit, up to NN_SMAX (bytes
// in flight per SM against DRAM latency: a load-only probe of 128-row x
// 16-column boxes over a 6.3M x 200 column-major matrix measured 5.4 TB/s
// with 4 stages, 6.3 TB/s with 7 to 12), at least 4.
int bres_stages(int ksteps, int Np) {
  int ns = NN_SMAX;
  while (ns > 4 && bres_smem(ksteps, Np, ns) > (size_t)kMaxSmem) --ns;
  return ns;
}
size_t ares_entry_bytes(int bn, int G) { return ((size_t)2 * G * bn * 32 + 1023) & ~(size_t)1023; }
size_t ares_smem(int bn, int sa, int nb, int G) {
  return 1024 + (size_t)sa * 8192 + (size_t)nb * ares_entry_bytes(bn, G) + AR_STG + 512;
}
// K-slices per B ring entry for (bn, sa, nb): the fewest entries per chunk
// (G = ceil(ks / E) for E = 1, 2, ...) whose nb entries fit in shared memory;
// 0 when not even single slices fit.
int ares_group(int ksteps, int bn, int sa, int nb) {
  for (int E = 1; E <= ksteps; ++E) {
    const int G = (ksteps + E - 1) / E;
    if (ares_smem(bn, sa, nb, G) <= (size_t)kMaxSmem) return G;
  }
  return 0;
}

struct AresCfg {
  int bn, sa, nb;
};
// Configuration override for tuning sweeps (bn = 0: automatic).
AresCfg g_ares_override = {0, 0, 0};
// Configurations chosen by the autotuner, per number of 16-wide k-slices.
AresCfg g_ares_tuned[AR_MAXKS + 1] = {};
std::mutex g_ares_mu;

// Default chunk width for N output columns: the least padded width
// (chunks x chunk width) among chunks of at least 128 columns (or N rounded
// up to 16, if smaller) up to the widest that fits, ties to the wider chunk.
// The products are bound by the tensor pipe's rate and by the issue cost per
// instruction together (measured at 6.3M rows and 1000 frames, 150 modes:
// 7 x 144 = 1008 columns 6.27 ms, 6 x 176 = 1056 6.3-6.4 ms, 8 x 128 = 1024
// 6.45 ms, 9 x 112 = 1008 6.40 ms).
int ares_bn(int ksteps, int N) {
  const int bmax = ares_bn_max(ksteps);
  const int bmin = (int)std::min<int64_t>(bmax, std::min<int64_t>(128, round_up(N, 16)));
  int best = bmax;
  int64_t best_w = ceil_div(N, bmax) * bmax;
  for (int bn = bmax - 16; bn >= bmin; bn -= 16) {
    const int64_t w = ceil_div(N, bn) * bn;
    if (w < best_w) {
      best = bn;
      best_w = w;
    }
  }
  return best;
}

// Default rings for chunk width bn: the most A stages (4 .. 2) with which
// any ring fits, then the fewest ring entries per chunk, then the most
// entries (measured at 6.3M rows, 1000 frames: 3 A stages better than 2 at
// every chunk width; 150 modes best with 3 entries of 5 K-slices, 200 modes
// with 2 entries of 7 and 6).  bn = 0 when nothing fits.
AresCfg ares_rings(int ksteps, int bn) {
  for (int sa = AR_MAXSA; sa >= 2; --sa) {
    AresCfg best = {0, 0, 0};
    int bestE = 1 << 30;
    for (int nb = AR_MAXNB; nb >= 2; --nb) {
      const int G = ares_group(ksteps, bn, sa, nb);
      if (G == 0) continue;
      const int E = (ksteps + G - 1) / G;
      if (E < bestE) {
        best = {bn, sa, nb};
        bestE = E;
      }
    }
    if (best.bn) return best;
  }
  return {0, 0, 0};
}

// Tuned configuration if any, else the default chunk width and its rings
// (or the first narrower chunk whose rings fit).
AresCfg ares_cfg(int ksteps, int N) {
  if (g_ares_override.bn) return g_ares_override;
  if (ksteps >= 1 && ksteps <= AR_MAXKS) {
    std::lock_guard<std::mutex> lock(g_ares_mu);
    if (g_ares_tuned[ksteps].bn) return g_ares_tuned[ksteps];
  }
  for (int bn = ares_bn(ksteps, N); bn >= 16; bn -= 16) {
    const AresCfg c = ares_rings(ksteps, bn);
    if (c.bn) return c;
  }
  return {0, 0, 0};
}
size_t tn_smem(int Mt, int Np, int nsplit, int ns) {
  const size_t st = ((size_t)128 * Mt * 128 + (size_t)128 * Np + 1023) & ~(size_t)1023;
  const size_t cv = ((size_t)nsplit * (Mt * 128 * 32 + Np * 32) + 1023) & ~(size_t)1023;
  return 1024 + ns * st + 2 * cv + 256;
}
// Deepest TMA ring (2 .. TN_S stages) that fits in shared memory (0: none does).
int tn_stages(int Mt, int Np, int nsplit) {
  for (int ns = TN_S; ns >= 2; --ns)
    if (tn_smem(Mt, Np, nsplit, ns) <= (size_t)kMaxSmem) return ns;
  return 0;
}

// Largest column chunk of B that stays resident for the B-resident kernel.
int bres_cols(int ksteps) {
  int np = 256;
  while (np > 16 && bres_smem(ksteps, np, 4) > (size_t)kMaxSmem) np -= 16;
  return np;
}

// Flush segments of the tensor-core reductions.  A CTA sums its rows in FP32
// tensor memory (3 products per 16-row k-step) and adds the sum to its FP64
// partial every `flush` k-steps; the FP32 rounding of a segment grows with its
// length (measured on a 8192-row projection: 256-k-step segments cost 3x the
// error of the split itself, 32-k-step ones add little).  So segments are as
// short as the FP64 flushes allow: about 1536 over the whole matrix (the
// number at 6.3M rows with 256-k-step segments), between 16 and 256 k-steps,
// and the grid gives every CTA at least one whole segment.
int tn_flush(int64_t n) {
  return (int)std::max<int64_t>(16, std::min<int64_t>(256, ceil_div(n, 16 * 1536)));
}
int tn_grid(int64_t n) {
  const int64_t want = ceil_div(n, 16 * (int64_t)tn_flush(n));
  return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), want));
}

}  // namespace

// ---------------------------------------------------------------- launchers

size_t umma_nn_workspace_bytes(int64_t n, int Kd, int N) {
  (void)n;
  const int ksteps = (int)ceil_div(Kd, 16);
  // recon layout (64-column chunks) is the larger of the two layouts
  const int64_t nch = ceil_div(N, 16);   // smallest chunk width gives the largest padding
  const size_t ares = (size_t)nch * 2 * ksteps * 16 * 32 + (size_t)2 * ksteps * 256 * 32;
  const size_t bres = (size_t)2 * ksteps * round_up(N, 16) * 32 + 2 * ksteps * 256 * 32;
  return std::max(ares, bres) + 4096;
}

size_t umma_tn_workspace_bytes(int64_t n, int Ka, int N) {
  // per-CTA FP64 partials for every (Ka-chunk, N-chunk) sub-problem, reused
  return (size_t)tn_grid(n) * std::min(Ka, 256) * std::min(N, 256) * sizeof(double) + 4096;
}

dmd_status umma_gemm_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const double* B, float* C, int64_t ldc,
                        void* ws, cudaStream_t st, int spare_sms, const int32_t* skip) {
  if (n <= 0 || N <= 0) return DMD_OK;
  const int ksteps = (int)ceil_div(Kd, 16);
  const int64_t ntiles = ceil_div(n, 128);
  uint8_t* split = reinterpret_cast<uint8_t*>(ws);
  CUtensorMap mapA;
  DMD_TRY(make_map(&mapA, A, n, Kd, lda, 128, 16));
  const int Npmax = bres_cols(ksteps);
  // persistent CTAs, one per SM; `spare_sms` SMs are left to work running
  // beside this product on another stream
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms() - spare_sms, ntiles));
  if (N <= 256 && round_up(N, 16) <= Npmax) {
    const int Np = (int)round_up(N, 16);
    const int64_t work = (int64_t)Np * ksteps;
    k_split_b<<<(unsigned)ceil_div(work, 128), 128, 0, st>>>(Kd, N, B, Np, ksteps, 1, split, skip);
    DMD_LAUNCH_CHECK();
    const int ns = bres_stages(ksteps, Np);
    const size_t smem = bres_smem(ksteps, Np, ns);
    DMD_CUDA_TRY(cudaFuncSetAttribute(k_umma_nn_bres, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_umma_nn_bres<<<grid, NN_THREADS, smem, st>>>(mapA, split, C, ldc, n, N, Np, ksteps, ntiles, ns, status_word(),
                                                   skip);
    DMD_LAUNCH_CHECK();
    return DMD_OK;
  }
  // many output columns: A tile resident, B streamed in bn-column chunks
  const AresCfg cfg = ares_cfg(ksteps, N);
  const int bn = cfg.bn;
  const int G = bn > 0 && ksteps <= AR_MAXKS ? ares_group(ksteps, bn, cfg.sa, cfg.nb) : 0;
  if (bn == 0 || ksteps > AR_MAXKS || G == 0 || bn > ares_bn_max(ksteps)) {
    set_error("umma_gemm_nn: inner dimension %d too large for the resident-A layout", Kd);
    return DMD_EINVAL;
  }
  const size_t smem = ares_smem(bn, cfg.sa, cfg.nb, G);
  const int nchunks = (int)ceil_div(N, bn);
  const int64_t work = (int64_t)nchunks * bn * ksteps;
  k_split_b<<<(unsigned)ceil_div(work, 128), 128, 0, st>>>(Kd, N, B, bn, ksteps, nchunks, split, skip);
  DMD_LAUNCH_CHECK();
  CUtensorMap mapC;
  DMD_TRY(make_map(&mapC, C, n, N, ldc, 32, 16));
  DMD_CUDA_TRY(cudaFuncSetAttribute(k_umma_nn_ares<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_umma_nn_ares<0><<<grid, AR_THREADS, smem, st>>>(mapA, mapC, split, n, N, ksteps, bn, cfg.sa, cfg.nb, G, nchunks,
                                                     ntiles, nullptr, nullptr, 0.f, nullptr, status_word(), skip);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

int umma_loss_parts(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), ceil_div(n, 128))); }

// Streamed loss of the frames F = A B (A n x Kd tall, B Kd x N FP64), the
// frames never stored: part[0 .. *parts) receives each CTA's share of
// sum_j w_j sum_i rho(F_ij - tgt_i) (rho quadratic, or Huber with delta > 0).
dmd_status umma_loss_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const double* B, const float* tgt,
                        const double* w, float delta, double* part, int* parts, void* ws, cudaStream_t st) {
  const int ksteps = (int)ceil_div(Kd, 16);
  const int64_t ntiles = ceil_div(n, 128);
  // 128-frame chunks where they fit (two 64-column epilogue rounds; the loss
  // stores nothing, so the products alone bound it: measured at 256^3 x 3
  // and 2000 frames, 128-frame chunks 91 ms against 97 ms for 144), else the
  // default chunk width, narrower only where the chunks' weights would not
  // fit in the 4096-entry staging area
  AresCfg cfg = {0, 0, 0};
  if (ksteps <= AR_MAXKS && N > 128 && ares_bn_max(ksteps) >= 128 && ceil_div(N, 128) * 128 <= 4096)
    cfg = ares_rings(ksteps, 128);
  if (ksteps <= AR_MAXKS)
    for (int bn = ares_bn(ksteps, N); bn >= 16 && cfg.bn == 0; bn -= 16)
      if (ceil_div(N, bn) * bn <= 4096) cfg = ares_rings(ksteps, bn);
  const int bn = cfg.bn;
  const int G = bn ? ares_group(ksteps, bn, cfg.sa, cfg.nb) : 0;
  if (ksteps > AR_MAXKS) {
    set_error("umma_loss_nn: inner dimension %d too large for the resident-A layout", Kd);
    return DMD_EINVAL;
  }
  if (bn == 0) {
    set_error("umma_loss_nn: %d frames in one call (at most 4096: the weights are staged in shared memory)", N);
    return DMD_EINVAL;
  }
  CUtensorMap mapA;
  DMD_TRY(make_map(&mapA, A, n, Kd, lda, 128, 16));
  const int grid = umma_loss_parts(n);
  const size_t smem = ares_smem(bn, cfg.sa, cfg.nb, G);
  const int nchunks = (int)ceil_div(N, bn);
  const int64_t work = (int64_t)nchunks * bn * ksteps;
  uint8_t* split = reinterpret_cast<uint8_t*>(ws);
  k_split_b<<<(unsigned)ceil_div(work, 128), 128, 0, st>>>(Kd, N, B, bn, ksteps, nchunks, split);
  DMD_LAUNCH_CHECK();
  DMD_CUDA_TRY(cudaFuncSetAttribute(k_umma_nn_ares<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // no frames are stored: the output map argument is unused (the A map stands in)
  k_umma_nn_ares<1><<<grid, AR_THREADS, smem, st>>>(mapA, mapA, split, n, N, ksteps, bn, cfg.sa, cfg.nb, G, nchunks,
                                                     ntiles, tgt, w, delta, part, status_word(), nullptr);
  DMD_LAUNCH_CHECK();
  *parts = grid;
  return DMD_OK;
}

// Autotuner of the resident-A (many output columns) product: every
// (frame chunk, A stages, B ring entries) configuration that fits in shared memory
// is launched on the caller's operands -- one warm-up and two timed launches,
// CUDA events on `st` -- and the fastest is kept for this number of k-slices;
// later products with the same inner dimension use it.  Synchronises `st`.
dmd_status umma_tune_nn(int64_t n, int Kd, int N, const float* A, int64_t lda, const double* B, float* C, int64_t ldc,
                        void* ws, cudaStream_t st, int32_t* chosen) {
  const int ksteps = (int)ceil_div(Kd, 16);
  if (n <= 0 || N <= 256 || ksteps < 1 || ksteps > AR_MAXKS) {   // not a resident-A product
    if (chosen) chosen[0] = chosen[1] = chosen[2] = 0;
    return DMD_OK;
  }
  cudaEvent_t e0, e1;
  DMD_CUDA_TRY(cudaEventCreate(&e0));
  DMD_CUDA_TRY(cudaEventCreate(&e1));
  AresCfg best = {0, 0, 0};
  float best_ms = 0.f;
  dmd_status status = DMD_OK;
  for (int bn = ares_bn_max(ksteps); bn >= 64 && status == DMD_OK; bn -= 16)
    for (int nb = 2; nb <= AR_MAXNB && status == DMD_OK; ++nb)
      for (int sa = 2; sa <= AR_MAXSA && status == DMD_OK; ++sa) {
        if (ares_group(ksteps, bn, sa, nb) == 0) continue;
        g_ares_override = {bn, sa, nb};
        status = umma_gemm_nn(n, Kd, N, A, lda, B, C, ldc, ws, st, 0, nullptr);
        if (status != DMD_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) status = DMD_ECUDA;
        for (int r = 0; r < 2 && status == DMD_OK; ++r) status = umma_gemm_nn(n, Kd, N, A, lda, B, C, ldc, ws, st, 0, nullptr);
        if (status != DMD_OK) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          set_error("umma_tune_nn: event timing failed");
          status = DMD_ECUDA;
          break;
        }
        if (best.bn == 0 || ms < best_ms) {
          best = {bn, sa, nb};
          best_ms = ms;
        }
      }
  g_ares_override = {0, 0, 0};
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DMD_TRY(status);
  {
    std::lock_guard<std::mutex> lock(g_ares_mu);
    g_ares_tuned[ksteps] = best;
  }
  if (chosen) {
    chosen[0] = best.bn;
    chosen[1] = best.sa;
    chosen[2] = best.nb;
  }
  return DMD_OK;
}

// C (Ka x N, ld Ka) = A^T B; sub-problems of at most 256 x 256 so that the
// accumulators (Mt * Np columns) fit in 512 TMEM columns.
dmd_status umma_gemm_tn_flush(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B, int64_t ldb,
                              double* C, int nsplit, int flush, void* ws, cudaStream_t st, const int32_t* skip) {
  if (n <= 0 || Ka <= 0 || N <= 0) return DMD_OK;
  if (flush <= 0) flush = tn_flush(n);
  double* part = reinterpret_cast<double*>(ws);
  const int grid = tn_grid(n);
  const int64_t chunk = round_up(ceil_div(n, grid), 32);
  const bool sym = A == B && Ka == N && lda == ldb && Ka <= 256;
  // The MMA's M side is padded to 128 rows, its N side to 16 columns: put the
  // operand that pads less on the M side (then reduce into C transposed).
  const bool swap = !sym && Ka <= 256 && N <= 256 &&
                    round_up(N, 128) * round_up(Ka, 16) < round_up(Ka, 128) * round_up(N, 16);
  const float* Am = swap ? B : A;
  const float* Bm = swap ? A : B;
  const int64_t ldam = swap ? ldb : lda, ldbm = swap ? lda : ldb;
  const int Km = swap ? N : Ka, Nm = swap ? Ka : N;
  for (int a0 = 0; a0 < Km; a0 += 256) {
    const int ka = std::min(256, Km - a0);
    const int Mt = (int)ceil_div(ka, 128);
    for (int b0 = 0; b0 < Nm; b0 += 256) {
      const int nb = std::min(256, Nm - b0);
      const int Np = (int)round_up(nb, 16);
      CUtensorMap mA, mB;
      DMD_TRY(make_map(&mA, Am + (int64_t)a0 * ldam, n, ka, ldam, 32, Mt * 128, true));
      DMD_TRY(make_map(&mB, Bm + (int64_t)b0 * ldbm, n, nb, ldbm, 32, Np, true));
      const int ns = tn_stages(Mt, Np, nsplit);
      if (ns == 0) {
        set_error("umma_gemm_tn: %d x %d block with %d-way split does not fit in shared memory", ka, nb, nsplit);
        return DMD_EINVAL;
      }
      const size_t smem = tn_smem(Mt, Np, nsplit, ns);
      DMD_CUDA_TRY(cudaFuncSetAttribute(k_umma_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_umma_tn<<<grid, TN_THREADS, smem, st>>>(mA, mB, n, ka, nb, Mt, Np, nsplit, flush, sym ? 1 : 0, ns, chunk,
                                                part, status_word(), skip);
      DMD_LAUNCH_CHECK();
      // reduce into the (a0, b0) block of C (of C^T when swapped)
      const int64_t count = (int64_t)ka * nb;
      double* dst = swap ? C + (int64_t)a0 * Ka + b0 : C + (int64_t)b0 * Ka + a0;
      k_reduce_parts<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(ka, nb, grid, part, dst, Ka, swap ? 1 : 0,
                                                                     skip);
      DMD_LAUNCH_CHECK();
    }
  }
  return DMD_OK;
}

dmd_status umma_gemm_tn(int64_t n, int Ka, int N, const float* A, int64_t lda, const float* B, int64_t ldb, double* C,
                        int nsplit, void* ws, cudaStream_t st) {
  return umma_gemm_tn_flush(n, Ka, N, A, lda, B, ldb, C, nsplit, 0, ws, st, nullptr);
}

}  // namespace dmd
