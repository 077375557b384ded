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
// k_umma_loss_grad works on 128-frame groups.  For one group, every CTA walks
// its 128-row tiles of Phi_R and for each tile:
//   fwd   D (128 frames x 128 rows) = C_g^T Phi_tile^T        (tensor memory)
//   epi   one thread per frame: e = x - t, loss += w rho(e), g = w rho'(e),
//         g split into bf16 hi / lo and written back into tensor memory over
//         D as the A operand of the next product
//   bwd   dC_g^T (128 frames x r) += G^T Phi_tile                (tensor memory)
// with every product in the BF16x3 form (hi*hi + hi*lo + lo*hi, FP32
// accumulation).  D / G is double-buffered and the MMA thread issues
// fwd(t + 1) before bwd(t), so the tensor pipe works on the next tile while
// the epilogue turns the current one into G.  dC_g^T is drained into a
// per-CTA FP64 partial every 32 tiles (4096 rows) and at the end of the
// group; the partials are summed over CTAs in a fixed order afterwards, so
// the result is deterministic.  Phi_R is read once per frame group, the
// coefficient group once per CTA.
//
// One bf16 copy of the tile (hi and lo planes) serves both products: core
// matrices of 8 rows x 8 modes (16-byte rows of 8 consecutive modes), at
// (row / 8) * RS + (mode / 8) * 128 bytes with RS = 256 ks.  The forward
// product reads it as its B operand K-major (N = rows, K = modes: K-adjacent
// cores 128 B apart, 8-row groups RS apart), the backward product as its B
// operand MN-major (N = modes, K = rows: K-adjacent cores RS apart, 8-mode
// groups 128 B apart).  The copy is double-buffered, so converting the next
// tile overlaps the current tile's products.
//
// Tensor memory (512 columns x 128 lanes, lane = frame of the group):
//   [0, 8 ks)                    C_g^T hi as an A operand (ks = K-slices of r)
//   [80, 208), [208, 336)        D, then G, two buffers: the tile's rows
//                                0..63 and 64..127 are handled by separate
//                                epilogue warps, each writing G over its own
//                                64 D columns (hi of its four 16-row slices,
//                                then lo)
//   [336, 336 + 16 ks)           dC_g^T accumulator (FP32, r padded to 16 ks)
// C_g^T lo is an A operand in shared memory (K-major, the tile layout with
// frames for rows).  Shared memory also holds a TMA ring of FP32 Phi slices
// (128 rows x 16 modes), the two tile copies and the tile's targets.
//
// Roles (14 warps): 0 TMA producer, 1 MMA issuer, 2-5 converters (FP32 slice
// -> bf16 planes), 6-13 epilogue (frame = TMEM lane; two warps per lane
// quarter, one per half of the tile's rows).  Every wait is bounded
// (2 s); a wait that runs out aborts the CTA: roles leave their loops, the
// producer and the MMA issuer drain what they issued, TMEM is freed and the
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

constexpr int LG_THREADS = 448;   // 14 warps: producer, MMA issuer, 4 converters, 8 epilogue
constexpr int LG_MAXKS = 10;      // r <= 160
constexpr int LG_RING = 3;        // TMA stages of FP32 Phi slices (8 KB each): as many as fit
constexpr int LG_FLUSH = 32;      // tiles between FP64 drains of dC^T
constexpr uint32_t LG_COL_D = 80, LG_COL_DC = 336;   // D / G buffers at 80 and 208

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

// Row t's 16 modes of slice s, split into bf16 hi / lo, into the tile copy
// (planes `hi` and `lo`, 8-row groups RS bytes apart).
__device__ __forceinline__ void store_tile_row(const float* x, uint8_t* hi, uint8_t* lo, int t, int s, uint32_t RS) {
  const uint32_t off = (uint32_t)(t >> 3) * RS + (uint32_t)s * 256u + (uint32_t)(t & 7) * 16u;
  uint4 h0, l0, h1, l1;
  split8(x, h0, l0);
  split8(x + 8, h1, l1);
  *reinterpret_cast<uint4*>(hi + off) = h0;
  *reinterpret_cast<uint4*>(hi + off + 128) = h1;
  *reinterpret_cast<uint4*>(lo + off) = l0;
  *reinterpret_cast<uint4*>(lo + off + 128) = l1;
}

template <bool kHuber>
__global__ void __launch_bounds__(LG_THREADS, 1)
    k_umma_loss_grad(const __grid_constant__ CUtensorMap tmPhi, int64_t n, int r, int K, int ks,
                     const double* __restrict__ C, const float* __restrict__ tgt, const double* __restrict__ wgt,
                     float delta, int64_t ntiles, double* __restrict__ part, double* __restrict__ loss_part,
                     int32_t* err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1024(smraw);
  const int Np = 16 * ks;                                    // r padded to the K-slices
  const uint32_t RS = (uint32_t)ks * 256u;                   // one 8-row group of a tile-layout copy
  const uint32_t plane = 16u * RS;                           // 128 rows x 16 ks modes x 2 bytes
  uint8_t* ring = sm;                                        // LG_RING x 8 KB
  uint8_t* phi = ring + LG_RING * 8192;                      // 2 buffers x (hi plane, lo plane)
  uint8_t* ctlo = phi + 4 * plane;                           // C_g^T lo (frames x modes)
  float* tgs = reinterpret_cast<float*>(ctlo + plane);       // [2][128] targets of the tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(tgs + 2 * 128);
  uint64_t* full = bars;                          // [LG_RING] slice landed
  uint64_t* empty = full + LG_RING;               // [LG_RING] slice converted
  uint64_t* phi_full = empty + LG_RING;           // [2][LG_MAXKS] slice s of tile buffer b converted
  uint64_t* bwd_done = phi_full + 2 * LG_MAXKS;   // [2] the bwd MMAs of buffer b's tile finished
  uint64_t* fwd_done = bwd_done + 2;              // [2] the fwd MMAs of buffer b's tile finished
  uint64_t* g_full = fwd_done + 2;                // [2] G of buffer b's tile in TMEM
  uint64_t* tg_full = g_full + 2;                 // [2] targets of buffer b's tile in place
  uint64_t* ct_full = tg_full + 2;                // C_g^T of the group in place
  uint64_t* dc_full = ct_full + 1;                // dC^T ready to drain
  uint64_t* dc_free = dc_full + 1;                // dC^T drained
  uint64_t* tdown = dc_free + 1;
  double* red = reinterpret_cast<double*>(tdown + 1);   // 8 epilogue warps' loss sums
  uint32_t* tslot = reinterpret_cast<uint32_t*>(red + 8);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < LG_RING; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 128);
    }
    for (int i = 0; i < 2 * LG_MAXKS; ++i) mbar_init(&phi_full[i], 128);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bwd_done[i], 1);
      mbar_init(&fwd_done[i], 1);
      mbar_init(&g_full[i], 256);
      mbar_init(&tg_full[i], 256);
    }
    mbar_init(ct_full, 256);
    mbar_init(dc_full, 1);
    mbar_init(dc_free, 256);
    mbar_init(tdown, 1);
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
  // of all groups form one sequence u = 0, 1, ... (u & 1 selects the buffers)
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_tiles * ngroups;
  auto drain_after = [&](int64_t u) {   // dC^T is drained after item u's bwd
    const int64_t j = u % my_tiles;
    return (j + 1) % LG_FLUSH == 0 || j + 1 == my_tiles;
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      uint32_t it = 0;
      bool issued[LG_RING];
      uint32_t par[LG_RING];
      for (int i = 0; i < LG_RING; ++i) issued[i] = false, par[i] = 0;
      bool ok = true;
      for (int64_t u = 0; ok && u < items; ++u) {
        const int64_t tile = blockIdx.x + (u % my_tiles) * gridDim.x;
        // the next item's tile into L2 now, so that its slices arrive from L2
        // when the ring (a few slices deep) asks for them
        if (u + 1 < items) {
          const int64_t nt = blockIdx.x + ((u + 1) % my_tiles) * gridDim.x;
          for (int s = 0; s < ks; ++s) tma_prefetch_2d(&tmPhi, (int)(nt * 128), s * 16);
        }
        for (int s = 0; s < ks; ++s, ++it) {
          const uint32_t st = it % LG_RING;
          if (!mbar_wait(&empty[st], ((it / LG_RING) & 1) ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[st], 8192);
          tma_load_2d(ring + st * 8192, &tmPhi, &full[st], (int)(tile * 128), s * 16);
          issued[st] = true;
          par[st] = (it / LG_RING) & 1;
        }
      }
      for (int i = 0; i < LG_RING; ++i)
        if (issued[i]) mbar_wait_drain(&full[i], par[i]);
    }
  } else if (warp == 1) {
    // -------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t id_fwd = idesc_bf16(128, 128);
      const uint32_t id_bwd = idesc_bf16(128, Np) | (1u << 16);   // B operand MN-major
      const uint64_t ctl0 = sdesc(su32(ctlo), 128u, RS);           // C_g^T lo, K-major
      uint32_t fl = 0;
      bool ok = true, fresh = true;
      // fwd(u): D of item u into buffer u & 1
      auto fwd = [&](int64_t u) -> bool {
        const uint32_t b = (uint32_t)(u & 1), use = (uint32_t)(u >> 1);
        if (u % my_tiles == 0) {   // first tile of a group: its coefficients must be in place
          if (!mbar_wait(ct_full, (uint32_t)(u / my_tiles) & 1, abort_flag)) return false;
          tc_after();
        }
        const uint8_t* hi = phi + b * 2 * plane;
        const uint64_t f0 = sdesc(su32(hi), 128u, RS), f_lo = plane >> 4;
        const uint32_t d = tmem + LG_COL_D + b * 128u;
        for (int s = 0; s < ks; ++s) {
          if (!mbar_wait(&phi_full[b * LG_MAXKS + s], use & 1, abort_flag)) return false;
          tc_after();
          const uint32_t ah = tmem + (uint32_t)s * 8u;
          const uint64_t al = ctl0 + (uint64_t)((uint32_t)s * 16u);
          const uint64_t bh = f0 + (uint64_t)((uint32_t)s * 16u), bl = bh + f_lo;
          umma_bf16_ta(d, ah, bh, id_fwd, s > 0 ? 1u : 0u);
          umma_bf16_ta(d, ah, bl, id_fwd, 1u);
          umma_bf16(d, al, bh, id_fwd, 1u);
        }
        umma_commit(&fwd_done[b]);
        return true;
      };
      // bwd(u): dC^T += G(u)^T Phi_tile(u)
      auto bwd = [&](int64_t u) -> bool {
        const uint32_t b = (uint32_t)(u & 1), use = (uint32_t)(u >> 1);
        if (!mbar_wait(&g_full[b], use & 1, abort_flag)) return false;
        tc_after();
        if (fresh && fl > 0) {   // the previous drain must have read dC^T
          if (!mbar_wait(dc_free, (fl - 1) & 1, abort_flag)) return false;
          tc_after();
        }
        const uint8_t* hi = phi + b * 2 * plane;
        const uint64_t b0 = sdesc(su32(hi), RS, 128u), f_lo = plane >> 4;   // MN-major: LBO along K, SBO along N
        const uint32_t dc = tmem + LG_COL_DC, g0 = tmem + LG_COL_D + b * 128u;
        for (int s = 0; s < 8; ++s) {
          // G of row slice s: in the D columns of its half, hi then lo
          const uint32_t gh = g0 + (uint32_t)(s >> 2) * 64u + (uint32_t)(s & 3) * 8u, gl = gh + 32u;
          const uint64_t bh = b0 + (uint64_t)((2u * (uint32_t)s * RS) >> 4), bl = bh + f_lo;
          umma_bf16_ta(dc, gh, bh, id_bwd, (fresh && s == 0) ? 0u : 1u);
          umma_bf16_ta(dc, gh, bl, id_bwd, 1u);
          umma_bf16_ta(dc, gl, bh, id_bwd, 1u);
        }
        fresh = false;
        umma_commit(&bwd_done[b]);
        if (drain_after(u)) {
          umma_commit(dc_full);
          ++fl;
          fresh = true;
        }
        return true;
      };
      // issue order fwd(0), then per item: fwd(u + 1) before bwd(u), except
      // across a group boundary, where the next group's coefficients are
      // loaded only after item u's drain
      if (items > 0) ok = fwd(0);
      for (int64_t u = 0; ok && u < items; ++u) {
        const bool next_same_group = u + 1 < items && (u + 1) % my_tiles != 0;
        if (next_same_group) ok = fwd(u + 1);
        ok = ok && bwd(u);
        if (ok && u + 1 < items && !next_same_group) ok = fwd(u + 1);
      }
      umma_commit(tdown);
      mbar_wait_drain(tdown, 0);
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------- converters
    const int t = threadIdx.x - 64;   // 0..127: row of the tile
    uint32_t it = 0;
    bool ok = true;
    for (int64_t u = 0; ok && u < items; ++u) {
      const uint32_t b = (uint32_t)(u & 1);
      // tile buffer b is free once the bwd MMAs of item u - 2 are done
      if (u >= 2 && !mbar_wait(&bwd_done[b], (uint32_t)((u >> 1) - 1) & 1, abort_flag)) break;
      uint8_t* hi = phi + b * 2 * plane;
      for (int s = 0; s < ks; ++s, ++it) {
        const uint32_t st = it % LG_RING;
        if (!mbar_wait(&full[st], (it / LG_RING) & 1, abort_flag)) {
          ok = false;
          break;
        }
        const float* src = reinterpret_cast<const float*>(ring + st * 8192);
        float x[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) x[c] = src[c * 128 + t];   // row t, modes 16 s + c
        store_tile_row(x, hi, hi + plane, t, s, RS);
        fence_async_smem();
        mbar_arrive(&empty[st]);
        mbar_arrive(&phi_full[b * LG_MAXKS + s]);
      }
    }
  } else {
    // --------------------------------------------------------------- epilogue
    const int q = warp & 3;                                  // lane quarter (TMEM access rule)
    const int h = (warp - 6) >> 2;                           // half of the tile's rows: 0..63 / 64..127
    const int f = q * 32 + lane;                             // frame within the group = TMEM lane
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int s_lo = h * ((ks + 1) >> 1), s_hi = h ? ks : ((ks + 1) >> 1);   // coefficient slices of this half
    uint32_t fl = 0;
    bool ok = true;
    double lacc = 0.0;
    // the target of row f of the next item (loaded one item ahead by the
    // first half's threads, which fill the shared copy)
    auto target_of = [&](int64_t u) -> float {
      const int64_t row = (blockIdx.x + (u % my_tiles) * gridDim.x) * 128 + f;
      return row < n ? tgt[row] : 0.f;
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
        // C_g^T: lane f holds C[:, fr] split into bf16 hi (TMEM) and lo (shared memory)
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
          tmem_st8(tmem + (uint32_t)s * 8u + lane_base, hh);
          const uint32_t off = (uint32_t)(f >> 3) * RS + (uint32_t)s * 256u + (uint32_t)(f & 7) * 16u;
          *reinterpret_cast<uint4*>(ctlo + off) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
          *reinterpret_cast<uint4*>(ctlo + off + 128) = make_uint4(ll[4], ll[5], ll[6], ll[7]);
        }
        tmem_st_wait();
        fence_async_smem();
        tc_before();
        mbar_arrive(ct_full);
      }
      const uint32_t b = (uint32_t)(u & 1), use = (uint32_t)(u >> 1);
      float* tg = tgs + b * 128;
      if (h == 0) {
        tg[f] = tnext;
        if (u + 1 < items) tnext = target_of(u + 1);
      }
      mbar_arrive(&tg_full[b]);
      if (!mbar_wait(&tg_full[b], use & 1, abort_flag) || !mbar_wait(&fwd_done[b], use & 1, abort_flag)) {
        ok = false;
        break;
      }
      tc_after();
      // this half's 64 D columns (rows 64 h .. 64 h + 63 of the tile)
      const uint32_t dcol = tmem + LG_COL_D + b * 128u + (uint32_t)h * 64u + lane_base;
      uint32_t v[64];
#pragma unroll
      for (int s = 0; s < 4; ++s) tmem_ld16_nw(dcol + (uint32_t)s * 16u, v + 16 * s);
      tmem_ld_wait();
      const float* tgh = tg + h * 64;
      float s_loss = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
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
        // G of row slice 4 h + s over this half's D columns, which this
        // thread has loaded: hi at 8 s, lo at 32 + 8 s
        tmem_st8(dcol + (uint32_t)s * 8u, hh);
        tmem_st8(dcol + 32u + (uint32_t)s * 8u, ll);
      }
      lacc += kHuber ? (double)s_loss : 0.5 * (double)s_loss;
      tmem_st_wait();
      tc_before();
      mbar_arrive(&g_full[b]);
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
    if (lane == 0) red[warp - 6] = ws;
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
  return 1024 + (size_t)LG_RING * 8192 + 5 * 16 * (size_t)ks * 256 + 2 * 128 * 4 + 512;
}

int lg_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), ceil_div(n, 128))); }

}  // namespace

// ---------------------------------------------------------------- launchers

bool umma_loss_grad_supported(int r) { return r >= 1 && r <= 16 * LG_MAXKS; }

// Workspace of umma_loss_grad: the per-CTA FP64 partials of dC (grid x K x r).
size_t umma_loss_grad_workspace_bytes(int64_t n, int r, int K) {
  return (size_t)lg_grid(n) * (size_t)K * (size_t)r * sizeof(double) + 256;
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
  const int ks = (int)ceil_div(r, 16);
  const int64_t ntiles = ceil_div(n, 128);
  const int grid = lg_grid(n);
  CUtensorMap map;
  DMD_TRY(make_map(&map, Phi, n, r, ldPhi, 128, 16));
  const size_t smem = lg_smem(ks);
  double* part = reinterpret_cast<double*>(ws);
  auto kern = delta > 0.f ? k_umma_loss_grad<true> : k_umma_loss_grad<false>;
  DMD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, LG_THREADS, smem, st>>>(map, n, r, K, ks, C, tgt, w, delta, ntiles, part, loss_part,
                                                   nullptr);
  DMD_LAUNCH_CHECK();
  const int64_t count = (int64_t)K * r;
  k_reduce_dc<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, grid, part, dC);
  DMD_LAUNCH_CHECK();
  *parts = grid;
  return DMD_OK;
}

}  // namespace dmd
