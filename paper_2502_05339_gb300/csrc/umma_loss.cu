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
//         g split into bf16 hi / lo and written back into tensor memory as
//         the A operand of the next product
//   bwd   dC_g^T (128 frames x r) += G^T Phi_tile                (tensor memory)
// with every product in the BF16x3 form (hi*hi + hi*lo + lo*hi, FP32
// accumulation).  dC_g^T is drained into a per-CTA FP64 partial every 32 tiles
// (4096 rows) and at the end of the group; the partials are summed over CTAs
// in a fixed order afterwards, so the result is deterministic.  Phi_R is read
// once per frame group (its tile is loaded twice in a row, the second time
// from L2, to be split into the two shared-memory layouts the two products
// need), the coefficient group once per CTA.
//
// Tensor memory (512 columns x 128 lanes, lane = frame of the group):
//   [0, 16 ks)            C_g^T as the A operand (bf16 hi, then lo; ks = K-slices of r)
//   [160, 288)            D, then G hi (8 row slices x 8 columns)
//   [288, 288 + 16 ks)    dC_g^T accumulator (FP32, r padded to 16 ks columns)
//   [448, 512)            G lo
// Shared memory: a TMA ring of FP32 Phi slices (128 rows x 16 modes), Phi_tile
// as the fwd B operand (N = rows, K = modes) and as the bwd B operand (N =
// modes, K = rows), both K-major without swizzle, and the tile's targets.
//
// Roles (10 warps): 0 TMA producer, 1 MMA issuer, 2-5 converters (FP32 slice
// -> bf16 planes), 6-9 epilogue (frame = TMEM lane).  Every wait is bounded
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

constexpr int LG_THREADS = 320;
constexpr int LG_MAXKS = 10;      // r <= 160
constexpr int LG_RING = 7;        // TMA stages of FP32 Phi slices (8 KB each): as many as fit
constexpr int LG_FLUSH = 32;      // tiles between FP64 drains of dC^T
constexpr uint32_t LG_COL_D = 160, LG_COL_DC = 288, LG_COL_GLO = 448;

__device__ __forceinline__ float rho_of(float e, float delta) {
  const float ae = fabsf(e);
  return (delta > 0.f && ae > delta) ? delta * (ae - 0.5f * delta) : 0.5f * e * e;
}
__device__ __forceinline__ float drho_of(float e, float delta) {
  return (delta > 0.f && fabsf(e) > delta) ? copysignf(delta, e) : e;
}

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

__global__ void __launch_bounds__(LG_THREADS, 1)
    k_umma_loss_grad(const __grid_constant__ CUtensorMap tmPhi, int64_t n, int r, int K, int ks,
                     const double* __restrict__ C, const float* __restrict__ tgt, const double* __restrict__ wgt,
                     float delta, int64_t ntiles, double* __restrict__ part, double* __restrict__ loss_part,
                     int32_t* err) {
  extern __shared__ uint8_t smraw[];
  uint8_t* sm = align1024(smraw);
  const int Np = 16 * ks;                                    // r padded to the K-slices
  const uint32_t fwd_plane = (uint32_t)ks * 4096u;           // ks slices x 128 rows x 32 B
  const uint32_t bwd_slice = (uint32_t)Np * 32u;             // one 16-row K-slice, Np modes
  const uint32_t bwd_plane = 8u * bwd_slice;
  uint8_t* ring = sm;                                        // LG_RING x 8 KB
  uint8_t* phif = ring + LG_RING * 8192;                     // fwd B: hi plane, lo plane
  uint8_t* phib = phif + 2 * fwd_plane;                      // bwd B: hi plane, lo plane
  float* tgs = reinterpret_cast<float*>(phib + 2 * bwd_plane);   // 4 warps x 128 targets
  uint64_t* bars = reinterpret_cast<uint64_t*>(tgs + 4 * 128);
  uint64_t* full = bars;                          // [LG_RING] slice landed
  uint64_t* empty = full + LG_RING;               // [LG_RING] slice converted
  uint64_t* fwd_full = empty + LG_RING;           // [LG_MAXKS] fwd B slice s of the tile ready
  uint64_t* bwd_full = fwd_full + LG_MAXKS;       // whole bwd B of the tile ready
  uint64_t* fwd_done = bwd_full + 1;              // fwd MMAs of the tile finished
  uint64_t* g_full = fwd_done + 1;                // G of the tile in TMEM
  uint64_t* bwd_done = g_full + 1;                // bwd MMAs of the tile finished
  uint64_t* ct_full = bwd_done + 1;               // C_g^T of the group in TMEM
  uint64_t* dc_full = ct_full + 1;                // dC^T ready to drain
  uint64_t* dc_free = dc_full + 1;                // dC^T drained
  uint64_t* tdown = dc_free + 1;
  double* red = reinterpret_cast<double*>(tdown + 1);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(red + 4);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < LG_RING; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 128);
    }
    for (int i = 0; i < LG_MAXKS; ++i) mbar_init(&fwd_full[i], 128);
    mbar_init(bwd_full, 128);
    mbar_init(fwd_done, 1);
    mbar_init(g_full, 128);
    mbar_init(bwd_done, 1);
    mbar_init(ct_full, 128);
    mbar_init(dc_full, 1);
    mbar_init(dc_free, 128);
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
  // flushes per group: after every LG_FLUSH tiles and after the group's last tile
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      uint32_t it = 0;
      bool issued[LG_RING];
      uint32_t par[LG_RING];
      for (int i = 0; i < LG_RING; ++i) issued[i] = false, par[i] = 0;
      bool ok = true;
      for (int g = 0; ok && g < ngroups; ++g)
        for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x)
          for (int pass = 0; ok && pass < 2; ++pass)
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
      for (int i = 0; i < LG_RING; ++i)
        if (issued[i]) mbar_wait_drain(&full[i], par[i]);
    }
  } else if (warp == 1) {
    // -------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t id_fwd = idesc_bf16(128, 128), id_bwd = idesc_bf16(128, Np);
      const uint64_t f0 = sdesc(su32(phif), kLBO, kSBO), b0 = sdesc(su32(phib), kLBO, kSBO);
      const uint64_t f_lo = fwd_plane >> 4, b_lo = bwd_plane >> 4;
      const uint32_t ct_lo = (uint32_t)ks * 8u;
      uint32_t tit = 0, fl = 0;
      bool ok = true;
      for (int g = 0; ok && g < ngroups; ++g) {
        if (!mbar_wait(ct_full, g & 1, abort_flag)) break;
        tc_after();
        int64_t j = 0;
        bool fresh = true;
        for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tit, ++j) {
          // D / G hi must be free: the previous tile's bwd MMAs have read G
          if (tit > 0 && !mbar_wait(bwd_done, (tit - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_after();
          for (int s = 0; s < ks; ++s) {
            if (!mbar_wait(&fwd_full[s], tit & 1, abort_flag)) {
              ok = false;
              break;
            }
            tc_after();
            const uint32_t ah = tmem + (uint32_t)s * 8u, al = ah + ct_lo;
            const uint64_t bh = f0 + (uint64_t)((uint32_t)s * 256u), bl = bh + f_lo;
            const uint32_t d = tmem + LG_COL_D;
            umma_bf16_ta(d, ah, bh, id_fwd, s > 0 ? 1u : 0u);
            umma_bf16_ta(d, ah, bl, id_fwd, 1u);
            umma_bf16_ta(d, al, bh, id_fwd, 1u);
          }
          if (!ok) break;
          umma_commit(fwd_done);
          if (!mbar_wait(g_full, tit & 1, abort_flag) || !mbar_wait(bwd_full, tit & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_after();
          if (fresh && fl > 0) {   // the previous drain must have read dC^T
            if (!mbar_wait(dc_free, (fl - 1) & 1, abort_flag)) {
              ok = false;
              break;
            }
            tc_after();
          }
          const uint32_t dc = tmem + LG_COL_DC;
          for (int s = 0; s < 8; ++s) {
            const uint32_t gh = tmem + LG_COL_D + (uint32_t)s * 8u, gl = tmem + LG_COL_GLO + (uint32_t)s * 8u;
            const uint64_t bh = b0 + (uint64_t)(((uint32_t)s * bwd_slice) >> 4), bl = bh + b_lo;
            umma_bf16_ta(dc, gh, bh, id_bwd, (fresh && s == 0) ? 0u : 1u);
            umma_bf16_ta(dc, gh, bl, id_bwd, 1u);
            umma_bf16_ta(dc, gl, bh, id_bwd, 1u);
          }
          fresh = false;
          umma_commit(bwd_done);
          if ((j + 1) % LG_FLUSH == 0 || j + 1 == my_tiles) {
            umma_commit(dc_full);
            ++fl;
            fresh = true;
          }
        }
      }
      umma_commit(tdown);
      mbar_wait_drain(tdown, 0);
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------- converters
    const int t = threadIdx.x - 64;   // 0..127
    uint32_t it = 0, tit = 0;
    bool ok = true;
    for (int g = 0; ok && g < ngroups; ++g) {
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tit) {
        // fwd B copy free once the previous tile's fwd MMAs are done
        if (tit > 0 && !mbar_wait(fwd_done, (tit - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
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
          uint8_t* hi = phif + (uint32_t)s * 4096u;
          split_store_row(x, hi, hi + fwd_plane, t);
          fence_async_smem();
          mbar_arrive(&empty[st]);
          mbar_arrive(&fwd_full[s]);
        }
        if (!ok) break;
        // bwd B copy free once the previous tile's bwd MMAs are done
        if (tit > 0 && !mbar_wait(bwd_done, (tit - 1) & 1, abort_flag)) {
          ok = false;
          break;
        }
        for (int s = 0; s < ks; ++s, ++it) {
          const uint32_t st = it % LG_RING;
          if (!mbar_wait(&full[st], (it / LG_RING) & 1, abort_flag)) {
            ok = false;
            break;
          }
          const float* src = reinterpret_cast<const float*>(ring + st * 8192);
          // 16 modes x 16 groups of 8 rows: unit u = mode (u >> 4), row group (u & 15)
#pragma unroll
          for (int k2 = 0; k2 < 2; ++k2) {
            const int u = t + 128 * k2;
            const int jm = u >> 4, rg = u & 15;
            const float4 a = *reinterpret_cast<const float4*>(src + jm * 128 + rg * 8);
            const float4 b = *reinterpret_cast<const float4*>(src + jm * 128 + rg * 8 + 4);
            const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            uint4 h, l;
            split8(x, h, l);
            const uint32_t off = (uint32_t)(rg >> 1) * bwd_slice + kslice_off(s * 16 + jm, rg & 1);
            *reinterpret_cast<uint4*>(phib + off) = h;
            *reinterpret_cast<uint4*>(phib + bwd_plane + off) = l;
          }
          fence_async_smem();
          mbar_arrive(&empty[st]);
        }
        if (!ok) break;
        mbar_arrive(bwd_full);
      }
    }
  } else {
    // --------------------------------------------------------------- epilogue
    const int q = warp & 3;
    const int f = q * 32 + lane;                             // frame within the group = TMEM lane
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float* tg = tgs + q * 128;
    uint32_t tit = 0, fl = 0;
    bool ok = true;
    double lacc = 0.0;
    for (int g = 0; ok && g < ngroups; ++g) {
      const int fr = g * 128 + f;                            // frame index
      const bool f_ok = fr < K;
      const float w = f_ok ? (float)wgt[fr] : 0.f;
      // C_g^T into TMEM: lane f holds C[:, fr] split into bf16 hi / lo
      {
        const double* col = C + (int64_t)fr * r;
        for (int s = 0; s < ks; ++s) {
          uint32_t h[8], l[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int m0 = s * 16 + 2 * i;
            const double v0 = (f_ok && m0 < r) ? col[m0] : 0.0, v1 = (f_ok && m0 + 1 < r) ? col[m0 + 1] : 0.0;
            const __nv_bfloat16 h0 = __float2bfloat16_rn((float)v0), h1 = __float2bfloat16_rn((float)v1);
            h[i] = pack2(h0, h1);
            l[i] = pack2(__float2bfloat16_rn((float)(v0 - (double)__bfloat162float(h0))),
                         __float2bfloat16_rn((float)(v1 - (double)__bfloat162float(h1))));
          }
          tmem_st8(tmem + (uint32_t)s * 8u + lane_base, h);
          tmem_st8(tmem + (uint32_t)(ks + s) * 8u + lane_base, l);
        }
        tmem_st_wait();
        tc_before();
        mbar_arrive(ct_full);
      }
      int64_t j = 0;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++tit, ++j) {
        const int64_t row0 = tile * 128;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t row = row0 + lane + 32 * i;
          tg[lane + 32 * i] = row < n ? tgt[row] : 0.f;
        }
        __syncwarp();
        const int rows = (int)((n - row0) < 128 ? (n - row0) : 128);
        if (!mbar_wait(fwd_done, tit & 1, abort_flag)) {
          ok = false;
          break;
        }
        tc_after();
        float s_loss = 0.f;
        for (int s = 0; s < 8; ++s) {
          float v[16];
          tmem_ld16(tmem + LG_COL_D + (uint32_t)s * 16u + lane_base, v);
          uint32_t h[8], l[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            float gv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int tr = s * 16 + 2 * i + u;
              const float e = v[2 * i + u] - tg[tr];
              const bool live = f_ok && tr < rows;
              s_loss += live ? w * rho_of(e, delta) : 0.f;
              gv[u] = live ? w * drho_of(e, delta) : 0.f;
            }
            const __nv_bfloat16 h0 = __float2bfloat16_rn(gv[0]), h1 = __float2bfloat16_rn(gv[1]);
            h[i] = pack2(h0, h1);
            l[i] = pack2(__float2bfloat16_rn(gv[0] - __bfloat162float(h0)),
                         __float2bfloat16_rn(gv[1] - __bfloat162float(h1)));
          }
          // G hi of rows 16 s .. 16 s + 15 overwrites D columns 8 s .. 8 s + 7,
          // which this thread has already loaded (slices s / 2 <= s)
          tmem_st8(tmem + LG_COL_D + (uint32_t)s * 8u + lane_base, h);
          tmem_st8(tmem + LG_COL_GLO + (uint32_t)s * 8u + lane_base, l);
        }
        lacc += (double)s_loss;
        tmem_st_wait();
        tc_before();
        mbar_arrive(g_full);
        if ((j + 1) % LG_FLUSH == 0 || j + 1 == my_tiles) {
          // drain dC^T (lane f = frame, columns = modes) into this CTA's FP64 partial
          if (!mbar_wait(dc_full, fl & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_after();
          double* dst = part + ((int64_t)blockIdx.x * K + fr) * r;
          const bool first = j < LG_FLUSH;
          for (int s = 0; s < ks; ++s) {
            float v[16];
            tmem_ld16(tmem + LG_COL_DC + (uint32_t)s * 16u + lane_base, v);
            if (f_ok) {
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int m = s * 16 + c;
                if (m < r) dst[m] = first ? (double)v[c] : dst[m] + (double)v[c];
              }
            }
          }
          tc_before();
          mbar_arrive(dc_free);
          ++fl;
        }
      }
    }
    const double ws = warp_sum(lacc);
    if (lane == 0) red[q] = ws;
  }
  tc_before();
  __syncthreads();
  if (warp == 1) {
    tc_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
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
  const size_t Np = 16 * (size_t)ks;
  return 1024 + (size_t)LG_RING * 8192 + 2 * (size_t)ks * 4096 + 2 * 8 * Np * 32 + 4 * 128 * 4 + 512;
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
  DMD_CUDA_TRY(cudaFuncSetAttribute(k_umma_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_umma_loss_grad<<<grid, LG_THREADS, smem, st>>>(map, n, r, K, ks, C, tgt, w, delta, ntiles, part, loss_part,
                                                   nullptr);
  DMD_LAUNCH_CHECK();
  const int64_t count = (int64_t)K * r;
  k_reduce_dc<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, grid, part, dC);
  DMD_LAUNCH_CHECK();
  *parts = grid;
  return DMD_OK;
}

}  // namespace dmd
