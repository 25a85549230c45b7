// vopp_noalloc.cu -- a belief update that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a belief update: a
// real-time control loop whose memory plan was fixed at start-up, a process whose GPU
// memory is entirely reserved by another framework's caching allocator, or code running
// where an allocation's implicit device synchronisation is not acceptable.  For them,
// vopp_belief_update_noalloc runs the same SIR kernel as vopp_belief_update on particle
// arrays the caller owns, and takes the kernel's working memory (propagated particles,
// the FP64 CDF, ancestors, the status word) from one fixed device array compiled into the
// library instead of from an allocator.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "vopp.h"
#include "vopp_internal.h"

namespace {

// Largest particle count the static scratch serves, and the scratch itself: per particle
// 8 B propagated state, 4 B log weight, 8 B CDF entry, 4 B ancestor; plus the status word.
// CROWD's 60-byte states fit fewer particles: (kNoAllocScratchBytes - 5 * 256) / 76 = 20695.
constexpr int kNoAllocMaxParticles = 65536;
constexpr size_t kNoAllocScratchBytes =
    (size_t)kNoAllocMaxParticles * (8 + 4 + 8 + 4) + 256 * 5;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (looked up once per device, with that
// device current).  In host code the array's name is only a host-side stand-in.
int scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices)
    return vopp::set_error(VOPP_E_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return vopp::set_error(VOPP_E_CUDA, "cudaGetDevice failed");
    if (cudaSetDevice(device) != cudaSuccess) return vopp::set_error(VOPP_E_CUDA, "cudaSetDevice failed");
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    cudaSetDevice(prev);
    if (e != cudaSuccess || !p)
      return vopp::set_error(VOPP_E_CUDA, "cudaGetSymbolAddress of the static scratch failed");
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return VOPP_OK;
}

inline size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Restores the calling thread's current device when it goes out of scope.
struct DeviceGuard {
  int prev = 0;
  bool ok = false;
  DeviceGuard() { ok = cudaGetDevice(&prev) == cudaSuccess; }
  ~DeviceGuard() { if (ok) cudaSetDevice(prev); }
};

// VOPP_OK when p is device (or managed) memory that `device` owns; VOPP_E_INVALID otherwise.
int check_device_array(const void *p, int device, const char *name) {
  cudaPointerAttributes at;
  std::memset(&at, 0, sizeof at);
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();   // clear the (non-sticky) error so that later calls do not see it
    return vopp::set_error(VOPP_E_INVALID, name);
  }
  const bool on_device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  if (!on_device || at.device != device) {
    char msg[160];
    std::snprintf(msg, sizeof msg, "%s is not device memory of the model's GPU %d", name, device);
    return vopp::set_error(VOPP_E_INVALID, msg);
  }
  return VOPP_OK;
}

}  // namespace

extern "C" VOPP_API int vopp_belief_update_noalloc(const vopp_model *model, void *states,
                                                   float *log_weights, int32_t n,
                                                   int32_t action, const void *obs,
                                                   uint64_t seed, uint64_t t,
                                                   uintptr_t cuda_stream, int32_t *ancestors,
                                                   double *ess_out, int32_t *resampled_out) {
  if (!model || !states || !log_weights || !obs)
    return vopp::set_error(VOPP_E_INVALID, "NULL argument");
  const int kind = vopp::model_kind(model);
  // 32-bit words per particle state (the root layout): NAV2D 2, CROWD 15, GRID / TOY2 1
  const size_t words = kind == VOPP_NAV2D ? 2 : (kind == VOPP_CROWD ? 15 : 1);
  const size_t per = 4 * words + 4 + 8 + 4;
  const int nmax = (int)std::min<size_t>((size_t)kNoAllocMaxParticles,
                                         (kNoAllocScratchBytes - 256 * 5) / per);
  if (n < 1 || n > nmax)
    return vopp::set_error(VOPP_E_INVALID,
                           "n outside [1, the capacity of the static scratch] (65536 particles; "
                           "CROWD: 20695)");
  const int A = kind == VOPP_NAV2D ? 4 : (kind == VOPP_GRID ? 13 : (kind == VOPP_CROWD ? 5 : 2));
  if (action < 0 || action >= A) return vopp::set_error(VOPP_E_INVALID, "action out of range");
  const int device = vopp::model_device(model);
  void *base = nullptr;
  int rc = scratch_address(device, &base);
  if (rc) return rc;
  // the caller's particle arrays must be device memory of the model's GPU: a host or
  // another GPU's pointer would be written by the kernel (nothing is allocated to check)
  if ((rc = check_device_array(states, device, "states")) ||
      (rc = check_device_array(log_weights, device, "log_weights")) ||
      (ancestors && (rc = check_device_array(ancestors, device, "ancestors"))))
    return rc;
  DeviceGuard guard;   // the caller's current device is restored on every return below
  if (!guard.ok || cudaSetDevice(device) != cudaSuccess)
    return vopp::set_error(VOPP_E_CUDA, "cudaSetDevice failed");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);

  // carve the static array: propagated states | log weights | CDF | ancestors | status
  char *p = static_cast<char *>(base);
  const size_t N = (size_t)n;
  char *t_states = p;           p += up256(4 * words * N);
  float *t_lw = reinterpret_cast<float *>(p);  p += up256(4 * N);
  double *cdf = reinterpret_cast<double *>(p); p += up256(8 * N);
  int *anc = reinterpret_cast<int *>(p);       p += up256(4 * N);
  vopp::BeliefOut *dout = reinterpret_cast<vopp::BeliefOut *>(p);

  vopp::BeliefArgs B;
  std::memset(&B, 0, sizeof B);
  B.kind = kind;
  B.N = n;
  B.action = action;
  B.key0 = (uint32_t)seed;
  B.key1 = (uint32_t)(seed >> 32);
  B.t = t;
  if (kind == VOPP_NAV2D) {
    float *xy = static_cast<float *>(states);
    float *txy = reinterpret_cast<float *>(t_states);
    B.x = xy; B.y = xy + n; B.tx = txy; B.ty = txy + n;
    const float *o = static_cast<const float *>(obs);
    B.obs_f[0] = o[0];
    B.obs_f[1] = o[1];
  } else if (kind == VOPP_CROWD) {   // rows: x, y, 12 people coordinates, flags
    float *st = static_cast<float *>(states);
    float *tst = reinterpret_cast<float *>(t_states);
    B.x = st; B.y = st + n; B.pf = st + 2 * N; B.s = reinterpret_cast<int *>(st + 14 * N);
    B.tx = tst; B.ty = tst + n; B.tpf = tst + 2 * N; B.ts = reinterpret_cast<int *>(tst + 14 * N);
    B.obs_i = *static_cast<const int32_t *>(obs);
  } else {
    B.s = static_cast<int *>(states);
    B.ts = reinterpret_cast<int *>(t_states);
    B.obs_i = *static_cast<const int32_t *>(obs);
  }
  B.lw = log_weights;
  B.tlw = t_lw;
  B.cdf = cdf;
  B.anc = ancestors ? reinterpret_cast<int *>(ancestors) : anc;
  B.model = vopp::model_device_tables(model);
  B.out = dout;

  // the status word keeps the previous call's contents: clear it first
  if (cudaMemsetAsync(dout, 0, sizeof(vopp::BeliefOut), stream) != cudaSuccess)
    return vopp::set_error(VOPP_E_CUDA, "clearing the status word failed");
  if (vopp::launch_belief(B, stream) != cudaSuccess)
    return vopp::set_error(VOPP_E_CUDA, "belief kernel launch failed");
  vopp::BeliefOut h;
  if (cudaMemcpyAsync(&h, dout, sizeof h, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return vopp::set_error(VOPP_E_CUDA, "reading the status word failed");
  if (h.status) return vopp::set_error(VOPP_E_DEGENERATE, "observation has zero likelihood under every particle");
  if (ess_out) *ess_out = h.ess;
  if (resampled_out) *resampled_out = h.resampled;
  return VOPP_OK;
}
