// Gaussian test matrix of the randomized range finder (Sec. 4.3).
//
// The paper only says the sketch matrix is "randomly initialized"; we draw
// N(0,1) entries from the counter-based Philox4x32-10 generator (Salmon,
// Moraes, Dror, Shaw, SC'11) so every element is a pure function of
// (seed, index) and the matrix can be regenerated anywhere without state.
#include "common.cuh"

namespace dmd {

namespace {

constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;   // round multipliers
constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u; // key schedule increments
constexpr uint32_t kSketchStream = 0x0D3D0001u;

__device__ __forceinline__ uint4 philox_round(uint4 c, uint2 k) {
  const uint32_t lo0 = kMul0 * c.x, hi0 = __umulhi(kMul0, c.x);
  const uint32_t lo1 = kMul1 * c.z, hi1 = __umulhi(kMul1, c.z);
  return make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  c = philox_round(c, k);
#pragma unroll
  for (int i = 1; i < 10; ++i) {
    k.x += kWeyl0;
    k.y += kWeyl1;
    c = philox_round(c, k);
  }
  return c;
}

__global__ void k_philox_blocks(int64_t count, uint32_t stream_id, uint64_t key, uint32_t* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint4 r = philox4x32_10(
      make_uint4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), stream_id, 0u),
      make_uint2((uint32_t)key, (uint32_t)(key >> 32)));
  reinterpret_cast<uint4*>(out)[i] = r;
}

// u in (0, 1): (x + 1/2) 2^-32
__device__ __forceinline__ double unit_open(uint32_t x) {
  return ((double)x + 0.5) * 2.3283064365386963e-10;
}

__global__ void k_sketch(int m, int l, uint64_t seed, double* Om) {
  const int64_t total = (int64_t)m * l;
  const int64_t blk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (4 * blk >= total) return;
  const uint4 r = philox4x32_10(
      make_uint4((uint32_t)blk, (uint32_t)((uint64_t)blk >> 32), kSketchStream, 0u),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  // two Box-Muller pairs: (x, y) -> radius from x, angle 2 pi y
  const double ra = sqrt(-2.0 * log(unit_open(r.x)));
  const double rb = sqrt(-2.0 * log(unit_open(r.z)));
  double sa, ca, sb, cb;
  sincospi(2.0 * unit_open(r.y), &sa, &ca);
  sincospi(2.0 * unit_open(r.w), &sb, &cb);
  const double g[4] = {ra * ca, ra * sa, rb * cb, rb * sb};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int64_t e = 4 * blk + t;
    if (e < total) Om[e] = g[t];  // column-major m x l: element e = i + m j
  }
}

}  // namespace

dmd_status launch_sketch(int m, int l, uint64_t seed, double* Om, cudaStream_t st) {
  const int64_t blocks = ceil_div((int64_t)m * l, 4);
  k_sketch<<<(unsigned)ceil_div(blocks, 256), 256, 0, st>>>(m, l, seed, Om);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

dmd_status launch_philox_blocks(int64_t count, uint32_t sid, uint64_t key, uint32_t* out,
                                cudaStream_t st) {
  if (count <= 0) return DMD_OK;
  k_philox_blocks<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, sid, key, out);
  DMD_LAUNCH_CHECK();
  return DMD_OK;
}

}  // namespace dmd
