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
// layout of the tensor cores, tile by tile (below).  k_umma_loss_grad runs on
// CTA pairs (2-CTA clusters) and works on 256-frame groups: CTA c of a pair
// holds frames 128 c .. 128 c + 127 of the group in its tensor-memory lanes,
// and the even CTA issues every product once for both (M = 256).  For one
// group, each pair walks its 192-row tiles and for each tile:
//   load  each CTA its two views of the tile (below) by bulk copies straight
//         into its shared memory (no conversion on the SM)
//   fwd   D (256 frames x 192 rows) = C_g^T Phi_tile^T         (tensor memory)
//   epi   one thread per frame: e = x - t, loss += w rho(e), g = w rho'(e),
//         g split into bf16 hi / lo and written back into tensor memory over
//         D as the A operand of the backward product, one 48-row quarter at
//         a time
//   bwd   dC_g^T (256 frames x r) += G_k^T Phi_k, quarter by quarter,
//         each as soon as both CTAs have written its G           (tensor memory)
// with every product in the BF16x3 form (hi*hi + hi*lo + lo*hi, FP32
// accumulation).  A tcgen05.mma holds its issuing thread ~130-160 cycles
// (measured), more than the tensor pipe needs for these shapes, so the
// design minimises instructions per row: the pair form (M = 256) and the
// wide forward product (N = 192 rows) give 66 instructions per 192 rows and
// 256 frames; the forward and backward products are issued by two threads.
// The one D / G accumulator is overwritten by fwd(t + 1) once bwd(t) has
// finished; only the first quarter's epilogue is exposed.  Forward views are
// double-buffered (the copies of tile t + 2 go out when fwd(t) has
// finished), the backward view single-buffered (its copies for tile t + 1
// go out when bwd(t) has finished and land while fwd(t + 1) runs); the even
// CTA prefetches tile t + 2 into L2.  dC_g^T is drained into a per-pair FP64
// partial every 32 tiles and at the end of the group; the partials are
// summed over pairs in a fixed order afterwards, so the result is
// deterministic.  The split copy is read once per 256-frame group (each byte
// by both CTAs of a pair, the second read from L2), the coefficient group
// once per CTA.
//
// Split tile layout (ks = K-slices of r; a plane holds 2 ks groups of 8
// modes): for plane p (hi, lo) and row half h (rows 96 h .. 96 h + 95),
// 8-mode group g is 1536 contiguous bytes, row t's 8 modes (bf16) at t * 16,
// at ((p * 2 + h) * 2 ks + g) * 1536 within the tile.  The products split B
// between the CTAs of the pair along N, so CTA c keeps two views of a tile
// in its shared memory:
//   forward view: row half c, all mode groups (N = rows: the pair's B has
//     rows 0..95 from CTA 0, 96..191 from CTA 1), read K-major (K-adjacent
//     groups 1536 B apart, 8-row groups 128 B apart);
//   backward view: both row halves, mode groups c ks .. c ks + ks - 1
//     (N = modes: the first half from CTA 0), read MN-major (K = rows: 8-row
//     groups 128 B apart, the second half 1536 ks B on; N: groups 1536 B
//     apart).
// Each view is one contiguous run (forward) or two (backward) of the tile.
//
// Tensor memory (512 columns x 128 lanes per CTA, lane = frame of its half
// of the group), allocated for the pair:
//   [0, 8 ks), [80, 80 + 8 ks)   C_g^T hi and lo as A operands
//   [160, 352)                   D, then G: quarter k (rows 48 k ..) in
//                                columns 48 k ..: hi of its three 16-row
//                                slices, then lo
//   [352, 352 + 16 ks)           dC_g^T accumulator (FP32, r padded to 16 ks)
//
// Roles (11 warps per CTA): 0 producer (bulk copies into its own CTA), 1 the
// forward MMA issuer (even CTA) or the relay that tells the even CTA when
// the odd CTA's views have landed, 2-9 epilogue (frame = TMEM lane; two
// warps per lane quarter, one for row quarters 0 and 2, one for 1 and 3;
// they arrive on the even CTA's barriers), 10 the backward MMA issuer (even
// CTA).  The products' completions arrive on the barriers of both CTAs.
// Every wait is bounded (2 s); a wait that runs out aborts the CTA: roles
// leave their loops, the producer and the issuers drain what they issued,
// the pair meets at a cluster barrier, tensor memory is freed and the
// status word gets DMD_ETIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace dmd {

int num_sms();

namespace {

constexpr int LG_THREADS = 352;   // 11 warps: producer, fwd issuer / relay, 8 epilogue, bwd issuer
constexpr int LG_WARP_BWD = 10;   // the warp that issues the backward products
constexpr int LG_MAXKS = 10;      // r <= 160
constexpr int LG_FLUSH = 32;      // tiles between FP64 drains of dC^T
constexpr int LG_TR = 192;        // rows of a tile
constexpr int LG_FRAMES = 256;    // frames of a group (128 per CTA of the pair)
constexpr uint32_t LG_HALF = LG_TR / 2;   // rows of a row half (a forward view)
constexpr uint32_t LG_QR = 48;            // rows (D columns) of a quarter: the unit of G and of bwd
constexpr int LG_NQ = LG_TR / LG_QR;      // quarters of a tile
constexpr int LG_QS = LG_QR / 16;         // 16-row k-steps per quarter
// tensor-memory columns: C_g^T hi, C_g^T lo, one D / G accumulator, dC_g^T
constexpr uint32_t LG_COL_CTHI = 0, LG_COL_CTLO = 8 * LG_MAXKS, LG_COL_D = 16 * LG_MAXKS,
                   LG_COL_DC = LG_COL_D + LG_TR;
static_assert(LG_COL_DC + 16 * LG_MAXKS <= 512, "tensor-memory layout exceeds 512 columns");
constexpr uint32_t LG_GROUP = LG_HALF * 16;  // bytes of one 8-mode group of a row half

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
// one thread per (tile, row half, 8-mode group, row); zeros past n and past r.
__global__ void k_split_phi(int64_t n, int r, int G, const float* __restrict__ Phi, int64_t ldPhi, int64_t ntiles,
                            uint8_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // (((tile * 2) + h) * G + g) * 48 + t
  if (i >= ntiles * 2 * G * (int64_t)LG_HALF) return;
  const int t = (int)(i % LG_HALF);
  const int64_t q = i / LG_HALF;
  const int g = (int)(q % G);
  const int64_t th = q / G;
  const int h = (int)(th & 1);
  const int64_t tile = th >> 1;
  const int64_t row = tile * LG_TR + h * (int64_t)LG_HALF + t;
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = g * 8 + c;
    x[c] = (row < n && j < r) ? Phi[(int64_t)j * ldPhi + row] : 0.f;
  }
  uint4 hi, lo;
  split8(x, hi, lo);
  const int64_t plane = 2 * (int64_t)G * LG_GROUP;   // both row halves
  uint8_t* dst = out + tile * 2 * plane + ((int64_t)h * G + g) * LG_GROUP + t * 16;
  *reinterpret_cast<uint4*>(dst) = hi;
  *reinterpret_cast<uint4*>(dst + plane) = lo;
}

template <bool kHuber>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(LG_THREADS, 1)
    k_umma_loss_grad(const uint8_t* __restrict__ tiles, int64_t n, int r, int K, int ks,
                     const double* __restrict__ C, const float* __restrict__ tgt, const double* __restrict__ wgt,
                     float delta, int64_t ntiles, double* __restrict__ part, double* __restrict__ loss_part,
                     int32_t* err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1024(smraw);
  const int Np = 16 * ks;                                    // r padded to the K-slices
  const int G = 2 * ks;                                      // 8-mode groups of r padded
  const uint32_t vplane = (uint32_t)G * LG_GROUP;            // one view plane (hi or lo)
  const uint32_t vsz = 2 * vplane;                           // one view (hi and lo planes)
  uint8_t* fview = sm;                                       // [2] forward views
  uint8_t* bview = sm + 2 * vsz;                             // the backward view
  float* tgs = reinterpret_cast<float*>(sm + 3 * vsz);       // [2][LG_TR] targets of the tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(tgs + 2 * LG_TR);
  uint64_t* fv_full = bars;                     // [2] this CTA's forward view b landed
  uint64_t* fv_peer = fv_full + 2;              // [2] (even CTA) the odd CTA's forward view b landed
  uint64_t* bv_full = fv_peer + 2;              // this CTA's backward view landed
  uint64_t* bv_peer = bv_full + 1;              // (even CTA) the odd CTA's backward view landed
  // one fwd completion barrier per forward-view buffer: with a single one,
  // fwd(u - 1) could complete before the producer looks for fwd(u - 2) and
  // the parity of the phase it waits for would come round again
  uint64_t* fwd_done = bv_peer + 1;             // [2] the fwd products of the item in view buffer b finished
  uint64_t* bwd_done = fwd_done + 2;            // the bwd products of the item finished
  uint64_t* g_full = bwd_done + 1;              // [LG_NQ] (even CTA) G of quarter k in both CTAs
  uint64_t* tg_full = g_full + LG_NQ;           // [2] targets of the item in place
  uint64_t* ct_full = tg_full + 2;              // (even CTA) C_g^T of the group in place in both CTAs
  uint64_t* dc_full = ct_full + 1;              // dC^T ready to drain
  uint64_t* dc_free = dc_full + 1;              // (even CTA) dC^T drained in both CTAs
  uint64_t* tdown = dc_free + 1;                // both issuers' products finished
  double* red = reinterpret_cast<double*>(tdown + 1);   // 8 epilogue warps' loss sums
  uint32_t* tslot = reinterpret_cast<uint32_t*>(red + 8);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t crank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
  const bool lead = crank == 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&fv_full[i], 1);
      mbar_init(&fv_peer[i], 1);
      mbar_init(&tg_full[i], 256);
    }
    mbar_init(bv_full, 1);
    mbar_init(bv_peer, 1);
    mbar_init(&fwd_done[0], 1);
    mbar_init(&fwd_done[1], 1);
    mbar_init(bwd_done, 1);
    for (int k = 0; k < LG_NQ; ++k) mbar_init(&g_full[k], 256);
    mbar_init(ct_full, 512);
    mbar_init(dc_full, 1);
    mbar_init(dc_free, 512);
    mbar_init(tdown, 2);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc_pair(tslot, 512);
  tc_before();
  __syncthreads();
  cluster_sync_all();   // both CTAs' barriers initialised before any remote arrival
  tc_after();
  const uint32_t tmem = *tslot;
  const int ngroups = (K + LG_FRAMES - 1) / LG_FRAMES;
  // tiles of this pair per group; a group's items are its tiles, and the
  // items of all groups form one sequence u = 0, 1, ...: item u uses forward
  // view buffer u & 1
  const int64_t pr = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int64_t my_tiles = ntiles > pr ? (ntiles - 1 - pr) / npairs + 1 : 0;
  const int64_t items = my_tiles * ngroups;
  const int64_t tile_bytes = 4 * (int64_t)vplane;
  auto tile_of = [&](int64_t u) { return pr + (u % my_tiles) * npairs; };
  auto drain_after = [&](int64_t u) {   // dC^T is drained after item u's bwd
    const int64_t j = u % my_tiles;
    return (j + 1) % LG_FLUSH == 0 || j + 1 == my_tiles;
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    // forward view of item u into buffer u & 1 once fwd(u - 2) has finished;
    // backward view of item u once bwd(u - 1) has finished
    if (lane == 0) {
      const uint32_t half = (uint32_t)ks * LG_GROUP;   // one row half of a backward view plane
      int64_t lastf[2] = {-1, -1}, lastb = -1;
      for (int64_t u = 0; u < items; ++u) {
        const uint32_t fb = (uint32_t)(u & 1);
        if (u >= 2 && !mbar_wait(&fwd_done[fb], (uint32_t)((u - 2) >> 1) & 1, abort_flag)) break;
        const uint8_t* src = tiles + tile_of(u) * tile_bytes;
        if (lead && u + 2 < items) bulk_prefetch_l2(tiles + tile_of(u + 2) * tile_bytes, 4 * vplane);
        mbar_expect_tx(&fv_full[fb], vsz);
        for (uint32_t p = 0; p < 2; ++p)   // row half crank, all mode groups
          bulk_g2s(fview + fb * vsz + p * vplane, src + p * 2 * vplane + crank * vplane, vplane, &fv_full[fb]);
        lastf[fb] = u;
        if (u >= 1 && !mbar_wait(bwd_done, (uint32_t)(u - 1) & 1, abort_flag)) break;
        mbar_expect_tx(bv_full, vsz);
        for (uint32_t p = 0; p < 2; ++p)   // mode groups crank ks .. of both row halves
          for (uint32_t h = 0; h < 2; ++h)
            bulk_g2s(bview + p * vplane + h * half, src + p * 2 * vplane + h * vplane + crank * half, half, bv_full);
        lastb = u;
      }
      // the copies in flight land before the CTA tears down
      for (int b = 0; b < 2; ++b)
        if (lastf[b] >= 0) mbar_wait_drain(&fv_full[b], (uint32_t)(lastf[b] >> 1) & 1);
      if (lastb >= 0) mbar_wait_drain(bv_full, (uint32_t)lastb & 1);
    }
  } else if (!lead && warp == 1) {
    // ---------------------------------------------- relay (odd CTA): views landed
    if (lane == 0) {
      for (int64_t u = 0; u < items; ++u) {
        const uint32_t fb = (uint32_t)(u & 1);
        if (!mbar_wait(&fv_full[fb], (uint32_t)(u >> 1) & 1, abort_flag)) break;
        mbar_arrive_remote(&fv_peer[fb], 0);
        if (!mbar_wait(bv_full, (uint32_t)u & 1, abort_flag)) break;
        mbar_arrive_remote(bv_peer, 0);
      }
    }
  } else if (lead && (warp == 1 || warp == LG_WARP_BWD)) {
    // ---------------------------------------------- MMA issuers (even CTA)
    // Two issuing threads, one per product; they order through barriers:
    // fwd(u) overwrites D / G once bwd(u - 1) has finished; bwd(u) reads G of
    // quarter k once both CTAs' epilogues have written it.
    if (lane == 0) {
      bool ok = true;
      if (warp == 1) {
        // fwd(u): D of item u; A = C_g^T (hi, lo) from tensor memory, B = the
        // forward views (K-major: K-adjacent 8-mode groups LG_GROUP apart,
        // 8-row groups 128 B apart)
        const uint32_t id_fwd = idesc_bf16(256, LG_TR);
        const uint32_t dcol = tmem + LG_COL_D;
        for (int64_t u = 0; ok && u < items; ++u) {
          const uint32_t fb = (uint32_t)(u & 1), use = (uint32_t)(u >> 1);
          if (u >= 1)
            if (!(ok = mbar_wait(bwd_done, (uint32_t)(u - 1) & 1, abort_flag))) break;
          if (u % my_tiles == 0)   // first tile of a group: both CTAs' coefficients in place
            if (!(ok = mbar_wait_cl(ct_full, (uint32_t)(u / my_tiles) & 1, abort_flag))) break;
          if (!(ok = mbar_wait(&fv_full[fb], use & 1, abort_flag) && mbar_wait_cl(&fv_peer[fb], use & 1, abort_flag)))
            break;
          tc_after();
          const uint64_t f0 = sdesc(su32(fview + fb * vsz), LG_GROUP, 128u), f_lo = vplane >> 4;
          for (int s = 0; s < ks; ++s) {
            const uint32_t ah = tmem + LG_COL_CTHI + (uint32_t)s * 8u, al = tmem + LG_COL_CTLO + (uint32_t)s * 8u;
            const uint64_t bh = f0 + (uint64_t)((uint32_t)s * (2u * LG_GROUP >> 4)), bl = bh + f_lo;
            umma_pair_ta(dcol, ah, bh, id_fwd, s > 0 ? 1u : 0u);
            umma_pair_ta(dcol, ah, bl, id_fwd, 1u);
            umma_pair_ta(dcol, al, bh, id_fwd, 1u);
          }
          umma_commit_pair(&fwd_done[fb]);
        }
      } else {
        // bwd(u), quarter by quarter: dC^T += G_k^T Phi_k; B = the backward
        // view (MN-major: K = rows, LBO, 8-row groups 128 B apart, the second
        // row half ks LG_GROUP on; N = modes, SBO, 8-mode groups LG_GROUP apart)
        const uint32_t id_bwd = idesc_bf16(256, Np) | (1u << 16);
        const uint32_t half = (uint32_t)ks * LG_GROUP;
        const uint32_t bv = su32(bview);
        const uint32_t dc = tmem + LG_COL_DC, g0 = tmem + LG_COL_D;
        uint32_t fl = 0;
        bool fresh = true;
        for (int64_t u = 0; ok && u < items; ++u) {
          if (!(ok = mbar_wait(bv_full, (uint32_t)u & 1, abort_flag) &&
                     mbar_wait_cl(bv_peer, (uint32_t)u & 1, abort_flag)))
            break;
          if (fresh && fl > 0)   // the previous drain must have read dC^T in both CTAs
            if (!(ok = mbar_wait_cl(dc_free, (fl - 1) & 1, abort_flag))) break;
          for (int k = 0; ok && k < LG_NQ; ++k) {
            if (!(ok = mbar_wait_cl(&g_full[k], (uint32_t)u & 1, abort_flag))) break;
            tc_after();
#pragma unroll
            for (int i = 0; i < LG_QS; ++i) {
              const int s = k * LG_QS + i;   // 16-row k-step of the tile
              // G of that slice: in quarter k's D columns, hi then lo
              const uint32_t gh = g0 + (uint32_t)k * LG_QR + (uint32_t)i * 8u, gl = gh + LG_QR / 2;
              const uint32_t hh = (uint32_t)(s * 16) / LG_HALF;                  // row half
              const uint32_t sa = bv + hh * half + ((uint32_t)(s * 16) % LG_HALF) / 8u * 128u;
              const uint64_t bh = sdesc(sa, 128u, LG_GROUP), bl = sdesc(sa + vplane, 128u, LG_GROUP);
              umma_pair_ta(dc, gh, bh, id_bwd, (fresh && s == 0) ? 0u : 1u);
              umma_pair_ta(dc, gh, bl, id_bwd, 1u);
              umma_pair_ta(dc, gl, bh, id_bwd, 1u);
            }
          }
          if (!ok) break;
          fresh = false;
          umma_commit_pair(bwd_done);
          if (drain_after(u)) {
            umma_commit_pair(dc_full);
            ++fl;
            fresh = true;
          }
        }
      }
      umma_commit_pair(tdown);   // one arrival per issuer in each CTA, when its products have finished
    }
  } else if (warp >= 2 && warp < 10) {
    // --------------------------------------------------------------- epilogue
    // Warp (lane quarter q, h) turns row quarters h and h + 2 into G, in
    // that order, so that quarters 0 and 1 are ready first.
    const int q = warp & 3;                                  // lane quarter (TMEM access rule)
    const int h = (warp - 2) >> 2;
    const int f = q * 32 + lane;                             // frame within this CTA's half = TMEM lane
    const int e = h * 128 + f;                               // this thread's row of the tile's targets
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int s_lo = h * ((ks + 1) >> 1), s_hi = h ? ks : ((ks + 1) >> 1);   // coefficient slices of this h
    uint32_t fl = 0;
    bool ok = true;
    double lacc = 0.0;
    // the target of row e of the next item (loaded one item ahead)
    auto target_of = [&](int64_t u) -> float {
      const int64_t row = tile_of(u) * LG_TR + e;
      return (e < LG_TR && row < n) ? tgt[row] : 0.f;
    };
    float tnext = items > 0 ? target_of(0) : 0.f;
    for (int64_t u = 0; ok && u < items; ++u) {
      const int g = (int)(u / my_tiles);
      const int64_t j = u % my_tiles;
      const int fr = g * LG_FRAMES + (int)crank * 128 + f;  // frame index
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
        mbar_arrive_remote(ct_full, 0);
      }
      const uint32_t d = (uint32_t)(u & 1), used = (uint32_t)(u >> 1);
      float* tg = tgs + d * LG_TR;
      if (e < LG_TR) tg[e] = tnext;
      if (u + 1 < items) tnext = target_of(u + 1);
      mbar_arrive(&tg_full[d]);
      if (!mbar_wait(&tg_full[d], used & 1, abort_flag) || !mbar_wait(&fwd_done[d], used & 1, abort_flag)) {
        ok = false;
        break;
      }
      tc_after();
      float s_loss = 0.f;
      for (int kk = 0; kk < 2; ++kk) {
        const int k = h + 2 * kk;                            // row quarter
        const uint32_t dcol = tmem + LG_COL_D + (uint32_t)k * LG_QR + lane_base;
        uint32_t v[LG_QR];
#pragma unroll
        for (int s = 0; s < LG_QS; ++s) tmem_ld16_nw(dcol + (uint32_t)s * 16u, v + 16 * s);
        tmem_ld_wait();
        const float* tgq = tg + k * LG_QR;
#pragma unroll
        for (int s = 0; s < LG_QS; ++s) {
          uint32_t hh[8], ll[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float2 tt = *reinterpret_cast<const float2*>(tgq + s * 16 + 2 * i);
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
          // G of slice s of quarter k over its D columns: hi at 8 s, lo at LG_QR / 2 + 8 s
          tmem_st8(dcol + (uint32_t)s * 8u, hh);
          tmem_st8(dcol + LG_QR / 2 + (uint32_t)s * 8u, ll);
        }
        tmem_st_wait();
        tc_before();
        mbar_arrive_remote(&g_full[k], 0);
      }
      lacc += kHuber ? (double)s_loss : 0.5 * (double)s_loss;
      if (drain_after(u)) {
        // drain dC^T (lane f = frame, columns = modes; this half's slices)
        // into the pair's FP64 partial
        if (!mbar_wait(dc_full, fl & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_after();
        double* dst = part + ((int64_t)pr * K + fr) * r;
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
        mbar_arrive_remote(dc_free, 0);
        ++fl;
      }
    }
    const double ws = warp_sum(lacc);
    if (lane == 0) red[warp - 2] = ws;
  }
  // teardown: the products (issued by the even CTA, reading both CTAs'
  // memories) have finished before either CTA frees its tensor memory or
  // leaves
  if (warp == 1 && lane == 0) mbar_wait_drain(tdown, 0);
  tc_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == 1) {
    tc_after();
    tmem_dealloc_pair(tmem, 512);
  }
  if (threadIdx.x == 0)
    loss_part[blockIdx.x] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
  if (threadIdx.x == 0 && *reinterpret_cast<volatile int*>(abort_flag)) raise_status(err, DMD_ETIMEOUT, 8004);
}

// dC[m + f r] = sum over pairs (fixed order) of part[pair][f][m].
__global__ void k_reduce_dc(int64_t count, int parts, const double* __restrict__ part, double* __restrict__ dC) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += part[(int64_t)p * count + i];
  dC[i] = s;
}

size_t lg_smem(int ks) {
  // two forward views and one backward view (hi and lo planes each), targets, barriers
  return 1024 + 3 * 2 * (size_t)(2 * ks) * LG_GROUP + 2 * LG_TR * 4 + 512;
}

// CTA pairs: one per two SMs, at most one per tile
int lg_pairs(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms() / 2, ceil_div(n, LG_TR))); }

size_t lg_part_bytes(int64_t n, int r, int K) {
  return (size_t)round_up((int64_t)lg_pairs(n) * K * r * (int64_t)sizeof(double), 1024);
}

size_t lg_split_bytes(int64_t n, int r) {
  const int64_t ks = ceil_div(r, 16);
  return (size_t)(ceil_div(n, LG_TR) * 4 * (2 * ks) * (int64_t)LG_GROUP);
}

}  // namespace

// ---------------------------------------------------------------- launchers

bool umma_loss_grad_supported(int r) { return r >= 1 && r <= 16 * LG_MAXKS; }

// Workspace of umma_loss_grad: the per-pair FP64 partials of dC (pairs x K x
// r) and the split tile copy of Phi_R (4 bytes per row and padded mode).
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
  const int pairs = lg_pairs(n);
  double* part = reinterpret_cast<double*>(ws);
  uint8_t* tiles = reinterpret_cast<uint8_t*>(ws) + lg_part_bytes(n, r, K);   // 1024-byte aligned
  const int64_t threads = ntiles * 2 * G * (int64_t)LG_HALF;
  k_split_phi<<<(unsigned)ceil_div(threads, 256), 256, 0, st>>>(n, r, G, Phi, ldPhi, ntiles, tiles);
  DMD_LAUNCH_CHECK();
  const size_t smem = lg_smem(ks);
  auto kern = delta > 0.f ? k_umma_loss_grad<true> : k_umma_loss_grad<false>;
  DMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<2 * pairs, LG_THREADS, smem, st>>>(tiles, n, r, K, ks, C, tgt, w, delta, ntiles, part, loss_part,
                                            status_word());
  DMD_LAUNCH_CHECK();
  const int64_t count = (int64_t)K * r;
  k_reduce_dc<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, pairs, part, dC);
  DMD_LAUNCH_CHECK();
  *parts = 2 * pairs;
  return DMD_OK;
}

}  // namespace dmd
