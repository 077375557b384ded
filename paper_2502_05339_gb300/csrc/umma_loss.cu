// Streamed per-frame loss and its gradient on the tensor cores (tcgen05,
// sm_103a), frames recomputed tile by tile and never written to memory.
//
// The objective of the prediction's adjoint (Sec. 7.2: gradients of the DMD
// operator for inverse design) is L = sum_j w_j sum_i rho(x_ij - t_i) over
// frames x_j = Phi_R C[:, j] and one target field t, with rho(e) = e^2 / 2 or
// the Huber function of width delta.  Its gradient with respect to the
// real-form coefficients is dC = Phi_R^T G with G_ij = w_j rho'(x_ij - t_i);
// the chain rule to lambda, beta (and the control inputs) is small FP64 work
// done elsewhere.
//
// k_split_phi first writes Phi_R once as bf16 hi / lo planes in the operand
// layout of the tensor cores, tile by tile (below); k_umma_loss_grad then
// works on 128-frame groups.  For one group, every CTA walks its 96-row tiles
// and for each tile:
//   load  the tile's hi and lo planes by bulk copies straight into shared
//         memory (no conversion on the SM)
//   fwd   D (128 frames x 96 rows) = C_g^T Phi_tile^T          (tensor memory)
//   epi   one thread per frame: e = x - t, loss += w rho(e), g = w rho'(e),
//         g split into bf16 hi / lo and written back into tensor memory over
//         D as the A operand of the next product
//   bwd   dC_g^T (128 frames x r) += G^T Phi_tile                (tensor memory)
// with every product in the BF16x3 form (hi*hi + hi*lo + lo*hi, FP32
// accumulation).  The forward and the backward products are issued by two
// threads: a tcgen05.mma holds its issuing thread ~130 cycles, about twice
// what the tensor pipe needs for these shapes, so one issuer leaves the pipe
// half idle.  D / G is double-buffered (fwd(t + 2) waits for bwd(t) to
// finish); three tile buffers let the copies of tile t + 3 go out as soon
// as bwd(t) has finished, and the producer prefetches that tile into L2
// three items ahead.  dC_g^T is drained into a
// per-CTA FP64 partial every 32 tiles and at the end of the group; the
// partials are summed over CTAs in a fixed order afterwards, so the result is
// deterministic.  The split copy is read once per frame group, the
// coefficient group once per CTA.
//
// Split tile layout (one plane = 2 ks groups of 8 modes, ks = K-slices of r):
// 8-mode group g of a 96-row tile is 1536 contiguous bytes, row t's 8 modes
// (bf16) at t * 16; groups follow each other, and a tile is its hi plane then
// its lo plane.  In shared memory the same bytes serve both products: the
// forward product reads them as its B operand K-major (N = rows: 8-row groups
// 128 B apart; K = modes: K-adjacent groups 1536 B apart), the backward
// product as its B operand MN-major (K = rows: 8-row groups 128 B apart;
// N = modes: 8-mode groups 1536 B apart).
//
// Tensor memory (512 columns x 128 lanes, lane = frame of the group):
//   [0, 8 ks), [80, 80 + 8 ks)   C_g^T hi and lo as A operands
//   [160, 256), [256, 352)       D, then G, two buffers: the tile's rows
//                                0..47 and 48..95 are handled by separate
//                                epilogue warps, each writing G over its own
//                                48 D columns (hi of its three 16-row slices,
//                                then lo)
//   [352, 352 + 16 ks)           dC_g^T accumulator (FP32, r padded to 16 ks)
//
// Roles (11 warps): 0 producer (bulk copies), 1 forward MMA issuer, 2-9
// epilogue (frame = TMEM lane; two warps per lane quarter, one per half of
// the tile's rows), 10 backward MMA issuer.  Every wait is bounded (2 s); a
// wait that runs out aborts the CTA: roles leave their loops, the producer
// and the MMA issuers drain what they issued, TMEM is freed and the status
// word gets DMD_ETIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace dmd {

int num_sms();

namespace {

constexpr int LG_THREADS = 352;   // 11 warps: producer, fwd issuer, 8 epilogue, bwd issuer
constexpr int LG_WARP_BWD = 10;   // the warp that issues the backward products
constexpr int LG_MAXKS = 10;      // r <= 160
constexpr int LG_FLUSH = 32;      // tiles between FP64 drains of dC^T
constexpr int LG_TR = 96;         // rows of a tile
constexpr int LG_NBUF = 3;        // tile buffers in shared memory
constexpr uint32_t LG_HALF = LG_TR / 2;   // rows (D columns) per epilogue half
constexpr int LG_HS = LG_TR / 32;         // 16-row slices per half
// tensor-memory columns: C_g^T hi, C_g^T lo, two D / G buffers, dC_g^T
constexpr uint32_t LG_COL_CTHI = 0, LG_COL_CTLO = 8 * LG_MAXKS, LG_COL_D = 16 * LG_MAXKS,
                   LG_COL_DC = LG_COL_D + 2 * LG_TR;
static_assert(LG_COL_DC + 16 * LG_MAXKS <= 512, "tensor-memory layout exceeds 512 columns");
constexpr uint32_t LG_GROUP = LG_TR * 16;  // bytes of one 8-mode group of a tile plane

// Split 8 consecutive FP32 values into bf16 hi / lo 16-byte chunks.
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]), h1 = __float2bfloat16_rn(x[2 * i + 1]);
    h[i] = pack2(h0, h1);
    l[i] = pack2(__float2bfloat16_rn(x[2 * i] - __bfloat162float(h0)),
                 __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1)));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Phi_R (n x r FP32, column-major, ld ldPhi) -> the split tile layout above:
// one thread per (tile, 8-mode group, row); zeros past n and past r.
__global__ void k_split_phi(int64_t n, int r, int G, const float* __restrict__ Phi, int64_t ldPhi, int64_t ntiles,
                            uint8_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // ((tile * G) + group) * LG_TR + row
  if (i >= ntiles * G * LG_TR) return;
  const int t = (int)(i % LG_TR);
  const int64_t tg = i / LG_TR;
  const int g = (int)(tg % G);
  const int64_t tile = tg / G;
  const int64_t row = tile * LG_TR + t;
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = g * 8 + c;
    x[c] = (row < n && j < r) ? Phi[(int64_t)j * ldPhi + row] : 0.f;
  }
  uint4 hi, lo;
  split8(x, hi, lo);
  uint8_t* dst = out + ((tile * 2) * G + g) * (int64_t)LG_GROUP + t * 16;
  *reinterpret_cast<uint4*>(dst) = hi;
  *reinterpret_cast<uint4*>(dst + (int64_t)G * LG_GROUP) = lo;
}

template <bool kHuber>
__global__ void __launch_bounds__(LG_THREADS, 1)
    k_umma_loss_grad(const uint8_t* __restrict__ tiles, int64_t n, int r, int K, int ks,
                     const double* __restrict__ C, const float* __restrict__ tgt, const double* __restrict__ wgt,
                     float delta, int64_t ntiles, double* __restrict__ part, double* __restrict__ loss_part,
                     int32_t* err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1024(smraw);
  const int Np = 16 * ks;                                    // r padded to the K-slices
  const uint32_t plane = (uint32_t)ks * 2u * LG_GROUP;       // one tile plane: LG_TR rows x 16 ks modes x 2 bytes
  uint8_t* phi = sm;                                         // LG_NBUF buffers x (hi plane, lo plane)
  float* tgs = reinterpret_cast<float*>(phi + 2 * LG_NBUF * plane);   // [2][LG_TR] targets of the tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(tgs + 2 * LG_TR);
  uint64_t* phi_full = bars;                           // [LG_NBUF][LG_MAXKS] slice s of tile buffer b landed
  uint64_t* bwd_done = phi_full + LG_NBUF * LG_MAXKS;  // [LG_NBUF] the bwd MMAs of tile buffer b's tile finished
  uint64_t* fwd_done = bwd_done + LG_NBUF;             // [2] the fwd MMAs into D / G buffer d finished
  uint64_t* g_full = fwd_done + 2;                     // [2] G in D / G buffer d
  uint64_t* tg_full = g_full + 2;                      // [2] targets of the item in place
  uint64_t* ct_full = tg_full + 2;                     // C_g^T of the group in place
  uint64_t* dc_full = ct_full + 1;                     // dC^T ready to drain
  uint64_t* dc_free = dc_full + 1;                     // dC^T drained
  uint64_t* tdown = dc_free + 1;
  double* red = reinterpret_cast<double*>(tdown + 1);   // 8 epilogue warps' loss sums
  uint32_t* tslot = reinterpret_cast<uint32_t*>(red + 8);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < LG_NBUF * LG_MAXKS; ++i) mbar_init(&phi_full[i], 1);
    for (int i = 0; i < LG_NBUF; ++i) mbar_init(&bwd_done[i], 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&fwd_done[i], 1);
      mbar_init(&g_full[i], 256);
      mbar_init(&tg_full[i], 256);
    }
    mbar_init(ct_full, 256);
    mbar_init(dc_full, 1);
    mbar_init(dc_free, 256);
    mbar_init(tdown, 2);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tslot, 512);
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = *tslot;
  const int ngroups = (K + 127) / 128;
  // tiles of this CTA per group; a group's items are its tiles, and the items
  // of all groups form one sequence u = 0, 1, ...: item u uses tile buffer
  // u % LG_NBUF and D / G buffer u & 1
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_tiles * ngroups;
  const int64_t tile_bytes = 2 * (int64_t)plane;
  auto tile_of = [&](int64_t u) { return blockIdx.x + (u % my_tiles) * gridDim.x; };
  auto drain_after = [&](int64_t u) {   // dC^T is drained after item u's bwd
    const int64_t j = u % my_tiles;
    return (j + 1) % LG_FLUSH == 0 || j + 1 == my_tiles;
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int64_t last[LG_NBUF];
      for (int b = 0; b < LG_NBUF; ++b) last[b] = -1;
      for (int64_t u = 0; u < items; ++u) {
        const uint32_t b = (uint32_t)(u % LG_NBUF), use = (uint32_t)(u / LG_NBUF);
        // tile buffer b is free once the bwd MMAs of item u - LG_NBUF are done
        if (u >= LG_NBUF && !mbar_wait(&bwd_done[b], (use - 1) & 1, abort_flag)) break;
        // the tile of item u + LG_NBUF into L2 now; its copies are issued LG_NBUF items later
        if (u + LG_NBUF < items) {
          const uint8_t* nx = tiles + tile_of(u + LG_NBUF) * tile_bytes;
          bulk_prefetch_l2(nx, plane);
          bulk_prefetch_l2(nx + plane, plane);
        }
        const uint8_t* src = tiles + tile_of(u) * tile_bytes;
        uint8_t* dst = phi + b * 2 * plane;
        for (int s = 0; s < ks; ++s) {
          uint64_t* bar = &phi_full[b * LG_MAXKS + s];
          mbar_expect_tx(bar, 2 * 2 * LG_GROUP);
          bulk_g2s(dst + s * 2 * LG_GROUP, src + s * 2 * LG_GROUP, 2 * LG_GROUP, bar);
          bulk_g2s(dst + plane + s * 2 * LG_GROUP, src + plane + s * 2 * LG_GROUP, 2 * LG_GROUP, bar);
        }
        last[b] = u;
      }
      // the copies in flight land before the CTA tears down
      for (int b = 0; b < LG_NBUF; ++b)
        if (last[b] >= 0)
          for (int s = 0; s < ks; ++s)
            mbar_wait_drain(&phi_full[b * LG_MAXKS + s], (uint32_t)(last[b] / LG_NBUF) & 1);
    }
  } else if (warp == 1 || warp == LG_WARP_BWD) {
    // ------------------------------------------------------------- MMA issuers
    // Two issuing threads, one per product: a tcgen05.mma holds its issuing
    // thread ~130 cycles (measured) while the tensor pipe runs it in about
    // half that, so one thread issuing both products would leave the pipe
    // idle.  The products order through barriers: fwd(u) overwrites D / G
    // buffer u & 1 once bwd(u - 2) has finished; bwd(u) reads G(u) once the
    // epilogue has written it.
    if (lane == 0) {
      bool ok = true;
      if (warp == 1) {
        // fwd(u): D of item u into D / G buffer u & 1; A = C_g^T (hi, lo)
        // from tensor memory, B = the tile K-major (K-adjacent 8-mode groups
        // LG_GROUP apart, 8-row groups 128 B apart)
        const uint32_t id_fwd = idesc_bf16(128, LG_TR);
        for (int64_t u = 0; ok && u < items; ++u) {
          const uint32_t tb = (uint32_t)(u % LG_NBUF), use = (uint32_t)(u / LG_NBUF), d = (uint32_t)(u & 1);
          if (u >= 2) {
            const int64_t p = u - 2;
            if (!(ok = mbar_wait(&bwd_done[p % LG_NBUF], (uint32_t)(p / LG_NBUF) & 1, abort_flag))) break;
            tc_after();
          }
          if (u % my_tiles == 0) {   // first tile of a group: its coefficients must be in place
            if (!(ok = mbar_wait(ct_full, (uint32_t)(u / my_tiles) & 1, abort_flag))) break;
            tc_after();
          }
          const uint64_t f0 = sdesc(su32(phi + tb * 2 * plane), LG_GROUP, 128u), f_lo = plane >> 4;
          const uint32_t dcol = tmem + LG_COL_D + d * LG_TR;
          for (int s = 0; s < ks; ++s) {
            if (!(ok = mbar_wait(&phi_full[tb * LG_MAXKS + s], use & 1, abort_flag))) break;
            tc_after();
            const uint32_t ah = tmem + LG_COL_CTHI + (uint32_t)s * 8u, al = tmem + LG_COL_CTLO + (uint32_t)s * 8u;
            const uint64_t bh = f0 + (uint64_t)((uint32_t)s * (2u * LG_GROUP >> 4)), bl = bh + f_lo;
            umma_bf16_ta(dcol, ah, bh, id_fwd, s > 0 ? 1u : 0u);
            umma_bf16_ta(dcol, ah, bl, id_fwd, 1u);
            umma_bf16_ta(dcol, al, bh, id_fwd, 1u);
          }
          if (ok) umma_commit(&fwd_done[d]);
        }
      } else {
        // bwd(u): dC^T += G(u)^T Phi_tile(u); B = the tile MN-major (K = rows:
        // LBO, 8-row groups 128 B apart; N = modes: SBO, 8-mode groups LG_GROUP apart)
        const uint32_t id_bwd = idesc_bf16(128, Np) | (1u << 16);
        uint32_t fl = 0;
        bool fresh = true;
        for (int64_t u = 0; ok && u < items; ++u) {
          const uint32_t tb = (uint32_t)(u % LG_NBUF), d = (uint32_t)(u & 1), used = (uint32_t)(u >> 1);
          if (!(ok = mbar_wait(&g_full[d], used & 1, abort_flag))) break;
          tc_after();
          if (fresh && fl > 0) {   // the previous drain must have read dC^T
            if (!(ok = mbar_wait(dc_free, (fl - 1) & 1, abort_flag))) break;
            tc_after();
          }
          const uint64_t b0 = sdesc(su32(phi + tb * 2 * plane), 128u, LG_GROUP), f_lo = plane >> 4;
          const uint32_t dc = tmem + LG_COL_DC, g0 = tmem + LG_COL_D + d * LG_TR;
#pragma unroll
          for (int s = 0; s < LG_TR / 16; ++s) {
            // G of row slice s: in the D columns of its half, hi then lo
            const uint32_t gh = g0 + (uint32_t)(s / LG_HS) * LG_HALF + (uint32_t)(s % LG_HS) * 8u;
            const uint32_t gl = gh + LG_HALF / 2;
            const uint64_t bh = b0 + (uint64_t)((uint32_t)s * (256u >> 4)), bl = bh + f_lo;
            umma_bf16_ta(dc, gh, bh, id_bwd, (fresh && s == 0) ? 0u : 1u);
            umma_bf16_ta(dc, gh, bl, id_bwd, 1u);
            umma_bf16_ta(dc, gl, bh, id_bwd, 1u);
          }
          fresh = false;
          umma_commit(&bwd_done[tb]);
          if (drain_after(u)) {
            umma_commit(dc_full);
            ++fl;
            fresh = true;
          }
        }
      }
      umma_commit(tdown);   // one arrival per issuer, when its products have finished
      mbar_wait_drain(tdown, 0);
    }
  } else {
    // --------------------------------------------------------------- epilogue
    const int q = warp & 3;                                  // lane quarter (TMEM access rule)
    const int h = (warp - 2) >> 2;                           // half of the tile's rows
    const int f = q * 32 + lane;                             // frame within the group = TMEM lane
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int s_lo = h * ((ks + 1) >> 1), s_hi = h ? ks : ((ks + 1) >> 1);   // coefficient slices of this half
    uint32_t fl = 0;
    bool ok = true;
    double lacc = 0.0;
    // the target of row f of the next item (loaded one item ahead by the
    // first half's threads, which fill the shared copy)
    auto target_of = [&](int64_t u) -> float {
      const int64_t row = tile_of(u) * LG_TR + f;
      return (f < LG_TR && row < n) ? tgt[row] : 0.f;
    };
    float tnext = (items > 0 && h == 0) ? target_of(0) : 0.f;
    for (int64_t u = 0; ok && u < items; ++u) {
      const int g = (int)(u / my_tiles);
      const int64_t j = u % my_tiles;
      const int fr = g * 128 + f;                            // frame index
      const bool f_ok = fr < K;
      // frames past K get weight 0, rows past n give e = 0 - 0 (zero-filled
      // Phi rows, zero targets): neither needs a mask below
      const float w = f_ok ? (float)wgt[fr] : 0.f;
      if (j == 0) {
        // C_g^T: lane f holds C[:, fr] split into bf16 hi and lo (tensor memory)
        const double* col = C + (int64_t)fr * r;
        for (int s = s_lo; s < s_hi; ++s) {
          uint32_t hh[8], ll[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int m0 = s * 16 + 2 * i;
            const double v0 = (f_ok && m0 < r) ? col[m0] : 0.0, v1 = (f_ok && m0 + 1 < r) ? col[m0 + 1] : 0.0;
            const __nv_bfloat16 h0 = __float2bfloat16_rn((float)v0), h1 = __float2bfloat16_rn((float)v1);
            hh[i] = pack2(h0, h1);
            ll[i] = pack2(__float2bfloat16_rn((float)(v0 - (double)__bfloat162float(h0))),
                          __float2bfloat16_rn((float)(v1 - (double)__bfloat162float(h1))));
          }
          tmem_st8(tmem + LG_COL_CTHI + (uint32_t)s * 8u + lane_base, hh);
          tmem_st8(tmem + LG_COL_CTLO + (uint32_t)s * 8u + lane_base, ll);
        }
        tmem_st_wait();
        tc_before();
        mbar_arrive(ct_full);
      }
      const uint32_t d = (uint32_t)(u & 1), used = (uint32_t)(u >> 1);
      float* tg = tgs + d * LG_TR;
      if (h == 0) {
        if (f < LG_TR) tg[f] = tnext;
        if (u + 1 < items) tnext = target_of(u + 1);
      }
      mbar_arrive(&tg_full[d]);
      if (!mbar_wait(&tg_full[d], used & 1, abort_flag) || !mbar_wait(&fwd_done[d], used & 1, abort_flag)) {
        ok = false;
        break;
      }
      tc_after();
      // this half's LG_HALF D columns (rows LG_HALF h .. of the tile)
      const uint32_t dcol = tmem + LG_COL_D + d * LG_TR + (uint32_t)h * LG_HALF + lane_base;
      uint32_t v[LG_HALF];
#pragma unroll
      for (int s = 0; s < LG_HS; ++s) tmem_ld16_nw(dcol + (uint32_t)s * 16u, v + 16 * s);
      tmem_ld_wait();
      const float* tgh = tg + h * LG_HALF;
      float s_loss = 0.f;
#pragma unroll
      for (int s = 0; s < LG_HS; ++s) {
        uint32_t hh[8], ll[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float2 tt = *reinterpret_cast<const float2*>(tgh + s * 16 + 2 * i);
          const float e0 = __uint_as_float(v[s * 16 + 2 * i]) - tt.x;
          const float e1 = __uint_as_float(v[s * 16 + 2 * i + 1]) - tt.y;
          float g0, g1;
          if (kHuber) {
            const float a0 = fabsf(e0), a1 = fabsf(e1);
            g0 = w * fminf(fmaxf(e0, -delta), delta);
            g1 = w * fminf(fmaxf(e1, -delta), delta);
            s_loss += w * (a0 > delta ? delta * (a0 - 0.5f * delta) : 0.5f * e0 * e0);
            s_loss += w * (a1 > delta ? delta * (a1 - 0.5f * delta) : 0.5f * e1 * e1);
          } else {
            g0 = w * e0;
            g1 = w * e1;
            s_loss = fmaf(g0, e0, s_loss);   // halved after the tile
            s_loss = fmaf(g1, e1, s_loss);
          }
          const __nv_bfloat162 hv = __floats2bfloat162_rn(g0, g1);
          const float2 hf = __bfloat1622float2(hv);
          const __nv_bfloat162 lv = __floats2bfloat162_rn(g0 - hf.x, g1 - hf.y);
          hh[i] = bf2_bits(hv);
          ll[i] = bf2_bits(lv);
        }
        // G of row slice LG_HS h + s over this half's D columns, which this
        // thread has loaded: hi at 8 s, lo at LG_HALF / 2 + 8 s
        tmem_st8(dcol + (uint32_t)s * 8u, hh);
        tmem_st8(dcol + LG_HALF / 2 + (uint32_t)s * 8u, ll);
      }
      lacc += kHuber ? (double)s_loss : 0.5 * (double)s_loss;
      tmem_st_wait();
      tc_before();
      mbar_arrive(&g_full[d]);
      if (drain_after(u)) {
        // drain dC^T (lane f = frame, columns = modes; this half's slices)
        // into this CTA's FP64 partial
        if (!mbar_wait(dc_full, fl & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_after();
        double* dst = part + ((int64_t)blockIdx.x * K + fr) * r;
        const bool first = j < LG_FLUSH;
        for (int s = s_lo; s < s_hi; ++s) {
          float dv[16];
          tmem_ld16(tmem + LG_COL_DC + (uint32_t)s * 16u + lane_base, dv);
          if (f_ok) {
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int m = s * 16 + c;
              if (m < r) dst[m] = first ? (double)dv[c] : dst[m] + (double)dv[c];
            }
          }
        }
        tc_before();
        mbar_arrive(dc_free);
        ++fl;
      }
    }
    const double ws = warp_sum(lacc);
    if (lane == 0) red[warp - 2] = ws;
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    tc_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0)
    loss_part[blockIdx.x] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(abort_flag)) raise_status(err, DMD_ETIMEOUT, 8004);
}

// dC[m + f r] = sum over CTAs (fixed order) of part[cta][f][m].
__global__ void k_reduce_dc(int64_t count, int parts, const double* __restrict__ part, double* __restrict__ dC) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += part[(int64_t)p * count + i];
  dC[i] = s;
}

size_t lg_smem(int ks) {
  // LG_NBUF tile buffers (hi + lo planes), targets, barriers
  return 1024 + 2 * LG_NBUF * (size_t)ks * 2 * LG_GROUP + 2 * LG_TR * 4 + 512;
}

int lg_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), ceil_div(n, LG_TR))); }

size_t lg_part_bytes(int64_t n, int r, int K) {
  return (size_t)round_up((int64_t)lg_grid(n) * K * r * (int64_t)sizeof(double), 1024);
}

size_t lg_split_bytes(int64_t n, int r) {
  const int64_t ks = ceil_div(r, 16);
  return (size_t)(ceil_div(n, LG_TR) * 2 * (2 * ks) * (int64_t)LG_GROUP);
}

}  // namespace

// ---------------------------------------------------------------- launchers

bool umma_loss_grad_supported(int r) { return r >= 1 && r <= 16 * LG_MAXKS; }

// Workspace of umma_loss_grad: the per-CTA FP64 partials of dC (grid x K x r)
// and the split tile copy of Phi_R (4 bytes per row and padded mode).
size_t umma_loss_grad_workspace_bytes(int64_t n, int r, int K) {
  return lg_part_bytes(n, r, K) + lg_split_bytes(n, r) + 256;
}

// loss_part[0 .. *parts) receives each CTA's loss; dC (r x K FP64) the
// gradient w.r.t. the coefficients C (r x K FP64, column-major).
dmd_status umma_loss_grad(int64_t n, int r, int K, const float* Phi, int64_t ldPhi, const double* C,
                          const float* tgt, const double* w, float delta, double* dC, double* loss_part, int* parts,
                          void* ws, cudaStream_t st) {
  if (!umma_loss_grad_supported(r)) {
    set_error("umma_loss_grad: r = %d outside 1..%d", r, 16 * LG_MAXKS);
    return DMD_EINVAL;
  }
  const int ks = (int)ceil_div(r, 16), G = 2 * ks;
  const int64_t ntiles = ceil_div(n, LG_TR);
  const int grid = lg_grid(n);
  double* part = reinterpret_cast<double*>(ws);
  uint8_t* tiles = reinterpret_cast<uint8_t*>(ws) + lg_part_bytes(n, r, K);   // 1024-byte aligned
  const int64_t threads = ntiles * G * LG_TR;
  k_split_phi<<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(n, r, G, Phi, ldPhi, ntiles, tiles);
  DMD_LAUNCH_CHECK();
  const size_t smem = lg_smem(ks);
  auto kern = delta > 0.f ? k_umma_loss_grad<true> : k_umma_loss_grad<false>;
  DMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, LG_THREADS, smem, st>>>(tiles, n, r, K, ks, C, tgt, w, delta, ntiles, part, loss_part,
                                       status_word());
  DMD_LAUNCH_CHECK();
  const int64_t count = (int64_t)K * r;
  k_reduce_dc<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, grid, part, dC);
  DMD_LAUNCH_CHECK();
  *parts = grid;
  return DMD_OK;
}

}  // namespace dmd
