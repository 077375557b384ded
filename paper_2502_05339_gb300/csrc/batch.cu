// Batched fit + predict of many scenes of uneven size (the many-scene
// workload of the method: each scene is an independent exact-DMD fit of its
// own snapshot matrix, Sec. 3.1 / Sec. 4.3, followed by the prediction of its
// frames, Eq. large_time_step).
//
// The fit of one scene is a chain of dependent launches; its tall passes fill
// the GPU only for large scenes, and its small FP64 solvers run on one or a
// few SMs.  The batch driver therefore runs scenes concurrently on `lanes`
// internal streams: scenes are assigned longest-first to the lane with the
// least accumulated work (n * m, a proxy of a scene's pass cost), each lane
// reuses one workspace sized for its largest scene (scenes on a lane run in
// order), and the lanes fork from and join back into the caller's stream
// through events.  Because the fork and join are stream-ordered, a call made
// while the caller's stream is being captured is captured whole, lanes
// included, so a batch can be replayed as one CUDA graph launch.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace dmd {
dmd_status predict_forward_workspace_bytes(const dmd_predict_desc* desc, size_t* bytes);
dmd_status predict_forward(const dmd_predict_desc* desc, const float* Phi_R, const double* modal, const int32_t* k,
                           const float* u, float* out, void* workspace, size_t ws_bytes, cudaStream_t st,
                           const char* who);
}  // namespace dmd

namespace {

constexpr int kMaxLanes = 32;
constexpr int kMaxDevices = 64;

struct LaneSet {
  cudaStream_t stream[kMaxLanes] = {};
  cudaEvent_t done[kMaxLanes] = {};
  cudaEvent_t fork = nullptr;
  bool ready = false;
};
std::mutex g_lane_mu;
LaneSet g_lanes[kMaxDevices];

dmd_status lanes_for_device(LaneSet** out) {
  int dev = 0;
  DMD_CUDA_TRY(cudaGetDevice(&dev));
  DMD_REQUIRE(dev >= 0 && dev < kMaxDevices, "dmd_fit_predict_batch: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_lane_mu);
  LaneSet& L = g_lanes[dev];
  if (!L.ready) {
    for (int i = 0; i < kMaxLanes; ++i) {
      DMD_CUDA_TRY(cudaStreamCreateWithFlags(&L.stream[i], cudaStreamNonBlocking));
      DMD_CUDA_TRY(cudaEventCreateWithFlags(&L.done[i], cudaEventDisableTiming));
    }
    DMD_CUDA_TRY(cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming));
    L.ready = true;
  }
  *out = &L;
  return DMD_OK;
}

dmd_predict_desc predict_desc_of(const dmd_scene& s) {
  dmd_predict_desc p{};
  p.n = s.fit.n;
  p.ldPhi = s.fit.ldPhi;
  p.ldOut = s.ldOut;
  p.r = s.fit.r;
  p.K = s.K;
  p.q = 0;
  p.steps = 0;
  p.precision = s.fit.precision;
  p.chunk = 0;
  return p;
}

dmd_status scene_bytes(const dmd_scene& s, size_t* bytes) {
  DMD_REQUIRE(s.fit.q == 0, "dmd_fit_predict_batch: scenes with control inputs are not batched");
  size_t fit = 0, pred = 0;
  DMD_TRY(dmd_fit_workspace_bytes(&s.fit, &fit));
  if (s.K > 0) {
    const dmd_predict_desc p = predict_desc_of(s);
    DMD_TRY(dmd::predict_forward_workspace_bytes(&p, &pred));
  }
  *bytes = (size_t)::dmd::round_up((int64_t)std::max(fit, pred), 256);
  return DMD_OK;
}

// Longest-first assignment to the least-loaded lane (deterministic).
void schedule(int count, const dmd_scene* scenes, int lanes, std::vector<int>& lane_of) {
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  auto cost = [&](int i) { return (double)scenes[i].fit.n * (double)(scenes[i].fit.m + 1); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<double> load(lanes, 0.0);
  lane_of.assign(count, 0);
  for (int i : order) {
    int best = 0;
    for (int l = 1; l < lanes; ++l)
      if (load[l] < load[best]) best = l;
    lane_of[i] = best;
    load[best] += cost(i);
  }
}

dmd_status lane_workspace(int count, const dmd_scene* scenes, int lanes, const std::vector<int>& lane_of,
                          std::vector<size_t>& lane_bytes) {
  lane_bytes.assign(lanes, 0);
  for (int i = 0; i < count; ++i) {
    size_t b = 0;
    DMD_TRY(scene_bytes(scenes[i], &b));
    lane_bytes[lane_of[i]] = std::max(lane_bytes[lane_of[i]], b);
  }
  return DMD_OK;
}

int clamp_lanes(int lanes, int count) {
  if (lanes <= 0) lanes = 16;
  return std::max(1, std::min({lanes, kMaxLanes, std::max(count, 1)}));
}

}  // namespace

extern "C" dmd_status dmd_batch_workspace_bytes(int32_t count, const dmd_scene* scenes, int32_t lanes,
                                                size_t* bytes) {
  DMD_REQUIRE(count >= 0 && (count == 0 || scenes != nullptr) && bytes != nullptr,
              "dmd_batch_workspace_bytes: bad arguments");
  lanes = clamp_lanes(lanes, count);
  std::vector<int> lane_of;
  schedule(count, scenes, lanes, lane_of);
  std::vector<size_t> lane_bytes;
  DMD_TRY(lane_workspace(count, scenes, lanes, lane_of, lane_bytes));
  size_t total = 0;
  for (size_t b : lane_bytes) total += b;
  *bytes = total + 256;
  return DMD_OK;
}

extern "C" dmd_status dmd_fit_predict_batch(int32_t count, const dmd_scene* scenes, int32_t lanes, void* workspace,
                                            size_t ws_bytes, void* stream) {
  DMD_REQUIRE(count >= 0 && (count == 0 || scenes != nullptr), "dmd_fit_predict_batch: bad scene array");
  if (count == 0) return DMD_OK;
  lanes = clamp_lanes(lanes, count);
  for (int i = 0; i < count; ++i) {
    const dmd_scene& s = scenes[i];
    DMD_REQUIRE(s.S && s.Phi_R && s.modal && s.info, "dmd_fit_predict_batch: scene %d has a NULL pointer", i);
    DMD_REQUIRE(s.K == 0 || (s.k && s.out && s.ldOut >= s.fit.n && s.ldOut % 4 == 0),
                "dmd_fit_predict_batch: scene %d: K > 0 needs k, out and ldOut >= n, a multiple of 4", i);
  }
  std::vector<int> lane_of;
  schedule(count, scenes, lanes, lane_of);
  std::vector<size_t> lane_bytes;
  DMD_TRY(lane_workspace(count, scenes, lanes, lane_of, lane_bytes));
  size_t total = 0;
  std::vector<size_t> lane_off(lanes, 0);
  for (int l = 0; l < lanes; ++l) {
    lane_off[l] = total;
    total += lane_bytes[l];
  }
  if (ws_bytes < total) {
    ::dmd::set_error("dmd_fit_predict_batch: workspace too small: %zu bytes given, %zu needed", ws_bytes, total);
    return DMD_ENOMEM;
  }
  DMD_REQUIRE(workspace != nullptr && ((uintptr_t)workspace & 255) == 0,
              "dmd_fit_predict_batch: workspace must be non-NULL and 256-byte aligned");
  LaneSet* L = nullptr;
  DMD_TRY(lanes_for_device(&L));
  cudaStream_t caller = (cudaStream_t)stream;
  DMD_CUDA_TRY(cudaEventRecord(L->fork, caller));
  for (int l = 0; l < lanes; ++l) DMD_CUDA_TRY(cudaStreamWaitEvent(L->stream[l], L->fork, 0));
  uint8_t* base = reinterpret_cast<uint8_t*>(workspace);
  // scenes in index order within each lane; the first failure stops the
  // enqueueing, and the lanes are joined back into the caller's stream
  // whatever happened, so that the caller's stream waits for every piece of
  // work already queued and a capture in progress stays well-formed
  dmd_status status = DMD_OK;
  for (int i = 0; i < count && status == DMD_OK; ++i) {
    const dmd_scene& s = scenes[i];
    const int l = lane_of[i];
    cudaStream_t st = L->stream[l];
    void* ws = base + lane_off[l];
    status = dmd_fit(&s.fit, s.S, nullptr, nullptr, s.Phi_R, s.modal, s.info, ws, lane_bytes[l], st);
    if (status == DMD_OK && s.K > 0) {
      const ::dmd::StatusScope scope(s.info);   // the scene's waits report to its own info
      const dmd_predict_desc p = predict_desc_of(s);
      status = ::dmd::predict_forward(&p, s.Phi_R, s.modal, s.k, nullptr, s.out, ws, lane_bytes[l], st,
                                      "dmd_fit_predict_batch");
    }
  }
  for (int l = 0; l < lanes; ++l) {
    const cudaError_t e1 = cudaEventRecord(L->done[l], L->stream[l]);
    const cudaError_t e2 = cudaStreamWaitEvent(caller, L->done[l], 0);
    if (status == DMD_OK && (e1 != cudaSuccess || e2 != cudaSuccess)) {
      ::dmd::set_error("dmd_fit_predict_batch: joining lane %d failed: %s", l,
                       cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
      status = DMD_ECUDA;
    }
  }
  return status;
}
