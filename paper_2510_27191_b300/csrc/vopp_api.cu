// vopp_api.cu -- host side of the libvopp C ABI (include/vopp.h).
//
// A context owns one CUDA stream handle, a device arena for tree storage (bounded by the
// HBM budget), a metadata block (plan descriptors, stage tables, results, root copies)
// mirrored in pinned host memory, and optional per-kernel event timing.  A plan call, or
// a batch of plans, is turned into a short sequence of launches -- root preparation, one
// materialising expansion per level, the fused leaf expansion, large-level backups and
// the per-plan tail with the FP64 root -- each launch covering every plan of the batch.
#include <algorithm>
#include <functional>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vopp.h"
#include "vopp_internal.h"

using namespace vopp;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CUDA_TRY(expr)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(VOPP_E_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));          \
  } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }


unsigned long long ipow(unsigned long long b, int e) {
  unsigned long long r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Timed kernel families; an expansion launch also counts under the level it writes
// ("expand_to_l<l>", every plan of the launch expanding into level l).
const char *kFamilies[] = {"root_prep", "expand", "leaf", "belief",
                           "expand_to_l1", "expand_to_l2", "expand_to_l3", "expand_to_l4",
                           "expand_to_l5", "expand_to_l6", "expand_to_l7", "expand_to_l8"};
enum { F_ROOT = 0, F_EXPAND, F_LEAF, F_BELIEF, F_COUNT };
constexpr int F_ALL = F_COUNT + kMaxDepth;
static_assert(sizeof(kFamilies) / sizeof(kFamilies[0]) == F_ALL, "one name per timed family");

struct TimedLaunch {
  int family;
  int level;           // expansions: the parent level (the launch writes level + 1)
  cudaEvent_t a, b;
};

}  // namespace

// ---------------------------------------------------------------------------------------
// Objects.
// ---------------------------------------------------------------------------------------
namespace {
// Resources of one in-flight launch sequence: its stream and a metadata block (plan
// descriptors, stage tables, results, root copies) in device memory with a pinned mirror.
struct Slot {
  cudaStream_t stream = nullptr;
  char *meta = nullptr;          // device metadata block
  char *hmeta = nullptr;         // pinned host mirror
  size_t meta_cap = 0;
  size_t off_res = 0, off_desc = 0;
  int n = 0;
};
}  // namespace

namespace {
// A captured launch sequence (metadata upload, every kernel, result download) of one batch
// shape, replayed while the shape, the buffers and the options stay the same.
// Instantiated launch sequences by signature (every launch shape, kernel parameter and
// buffer address the recorded operations bake in; the plans' tree pointers are not among
// them -- the kernels read those from the descriptors uploaded by the sequence itself).  At
// most kMaxGraphs are kept; the oldest is dropped first.
struct GraphSet {
  static constexpr size_t kMaxGraphs = 4096;
  std::unordered_map<std::string, cudaGraphExec_t> execs;
  std::deque<std::string> order;
  cudaStream_t capture = nullptr;   // private stream the sequence is recorded on (the legacy
                                    // default stream cannot be captured)
  void reset() {
    for (auto &kv : execs) cudaGraphExecDestroy(kv.second);
    execs.clear();
    order.clear();
  }
  void release() {
    reset();
    if (capture) cudaStreamDestroy(capture);
    capture = nullptr;
  }
};
struct Job;   // one plan of a launch sequence (below)
}  // namespace

struct vopp_ctx {
  int device = 0;
  int use_graphs = 0;            // replay captured launch sequences of repeated shapes
  GraphSet graph;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  char *arena = nullptr;
  size_t arena_cap = 0;
  Slot slot;                     // the synchronous path's slot (stream = ctx stream)
  bool plan_pending = false;     // vopp_plan_submit enqueued a plan; vopp_plan_finish collects
  std::vector<Job> pending_jobs;
  int leaf_persistent = 2;       // persistent leaf CTAs pulling work from a counter: 0 never,
                                 // 1 always, 2 per model (GRID and TOY2)
  int fp64_root = 0;             // root backup in FP64
  int sm_count = 148;
  int tree_detail = VOPP_TREE_MINIMAL;
  int leaf_gen = 1;              // generate level D-1 inside the leaf kernel
  int leaf_threads = 128;
  int grid_cap = 1 << 30;
  int reuse_copy = 1;            // plans continuing a kept subtree copy its levels (else recompute)
  int server_direct = 0;         // servers created now launch an idle server's requests at submit
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<TimedLaunch> pending;
  double fam_ms[F_ALL] = {0};
  unsigned long long fam_n[F_ALL] = {0};
  std::atomic<unsigned long long> h2d_bytes{0}, d2h_bytes{0}, launches{0};
  // last launch, for vopp_tree_read
  std::vector<PlanDesc> last_desc;
  std::vector<int> last_ok;
  EpisodeStore *episodes = nullptr;   // buffers of the last episode-mode plan
  // the library's stream-ordered pool (server arenas, kept trees, agents): memory stays in
  // it once allocated, and it never makes one stream wait for another to reuse memory
  cudaMemPool_t pool = nullptr;
};

struct vopp_model {
  vopp_ctx *ctx = nullptr;
  vopp_model_desc desc{};
  DevModel host{};
  DevModel *dev = nullptr;
  int A = 0;
};

struct vopp_env {
  vopp_model *model = nullptr;
  uint64_t seed = 0;
  unsigned long long t = 0;
  float *blk = nullptr;                 // the true state (one particle of the root layout)
  float *xy = nullptr;                  // NAV2D / CROWD robot (x, y)
  int *s = nullptr;                     // GRID / TOY2 state, CROWD flags
  float *pf = nullptr;                  // CROWD people
  EnvOut *dout = nullptr, *hout = nullptr;
};

struct KeptTree;   // a plan's tree kept on the device for subtree reuse (below)

struct vopp_agent {
  vopp_model *model = nullptr;
  int N = 0;
  uint64_t seed = 0;
  unsigned long long t = 0;
  // subtree reuse (vopp_agent_set_reuse): the last plan's tree, kept until the next plan or
  // belief update, and the subtree adopted by the last belief update, kept until the next
  int reuse = 0;
  KeptTree *tree = nullptr, *sub = nullptr;
  int adopted_slot = -1;                // branch a*W + k adopted by the last update, or -1
  // the memory of a released kept tree, for the agent's next plan (no allocation per plan):
  // taken once spare_ev, recorded after the last work that read it, has completed
  char *spare = nullptr;
  size_t spare_bytes = 0;
  cudaEvent_t spare_ev = nullptr;
  float *xy = nullptr, *lw = nullptr;   // NAV2D: xy[2N] (x then y)
  int *s = nullptr;                     // GRID / TOY2
  float *txy = nullptr, *tlw = nullptr;
  int *ts = nullptr;
  float *pf = nullptr, *tpf = nullptr;  // CROWD people [12][N]
  float *blk = nullptr, *tblk = nullptr;  // the state store (rows as the root layout)
  double *cdf = nullptr;
  int *anc = nullptr;
  BeliefOut *dout = nullptr;
  BeliefOut hout{};                     // host copy of the last update's outcome
};

// ---------------------------------------------------------------------------------------
// Plan layout in the arena.
// ---------------------------------------------------------------------------------------
namespace {

struct PlanShape {
  int kind, A, W, AW, N, D, pi_mode;
  int leaf_gen, keep_leaf, keep_debug, mat_top;
  int keep_obs;      // store the branch observations of every materialised level (kept trees)
};

struct PlanLayout {
  size_t bytes = 0;
  size_t px[kMaxDepth], py[kMaxDepth], plw[kMaxDepth], ps[kMaxDepth], pf[kMaxDepth];
  size_t rbar[kMaxDepth + 1], lom[kMaxDepth + 1], V[kMaxDepth + 1], Q[kMaxDepth],
      mu[kMaxDepth], rep[kMaxDepth + 1], obs[kMaxDepth + 1], cnt[kMaxDepth], psi[kMaxDepth];
};

constexpr size_t kNone = ~(size_t)0;

// 32-bit words per particle of the caller's root states (and of an agent's store).
size_t root_words(int kind) { return kind == kNav ? 2 : (kind == kCrowd ? 15 : 1); }

PlanShape make_shape(const vopp_model *m, int N, int D, int W, const vopp_ctx *ctx) {
  PlanShape s{};
  s.kind = m->desc.kind;
  s.A = m->A;
  s.W = W;
  s.AW = m->A * W;
  s.N = N;
  s.D = D;
  s.pi_mode = m->desc.pi_mode;
  s.leaf_gen = (D >= 2 && ctx->leaf_gen) ? 1 : 0;
  s.keep_debug = ctx->tree_detail == VOPP_TREE_FULL;
  s.keep_leaf = (ctx->tree_detail == VOPP_TREE_FULL || D == 1) ? 1 : 0;
  s.mat_top = (D == 0) ? 0 : (s.leaf_gen ? D - 2 : D - 1);
  return s;
}

// psi: also allocate the persistent preferences of every internal level (anytime plans).
PlanLayout make_layout(const PlanShape &s, bool psi = false) {
  PlanLayout L;
  for (int i = 0; i < kMaxDepth; ++i)
    L.px[i] = L.py[i] = L.plw[i] = L.ps[i] = L.pf[i] = L.Q[i] = L.mu[i] = L.cnt[i] = L.psi[i] = kNone;
  for (int i = 0; i <= kMaxDepth; ++i) L.rbar[i] = L.lom[i] = L.V[i] = L.rep[i] = L.obs[i] = kNone;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  for (int l = 0; l <= s.mat_top; ++l) {
    const size_t n = (size_t)ipow(s.AW, l) * (size_t)s.N;
    if (s.kind == kNav || s.kind == kCrowd) { L.px[l] = take(4 * n); L.py[l] = take(4 * n); }
    if (s.kind != kNav) L.ps[l] = take(4 * n);
    if (s.kind == kCrowd) L.pf[l] = take(48 * n);
    L.plw[l] = take(4 * n);
  }
  for (int l = 0; l <= s.D; ++l) {
    const size_t nodes = (size_t)ipow(s.AW, l);
    const bool node_level = l < s.D || s.D == 0;   // depth 0: the root holds V and Q
    const bool keep = node_level || s.keep_leaf;
    if (keep) L.V[l] = take(4 * nodes);
    if (node_level) L.Q[l] = take(4 * nodes * s.A);
    if (node_level && s.pi_mode == kPiNavDist) L.mu[l] = take(8 * nodes);
    if (l <= s.D - 2) L.cnt[l] = take(4 * nodes);
    if (psi && l < s.D) L.psi[l] = take(4 * nodes * s.A);
    if (l >= 1 && keep) { L.rbar[l] = take(4 * nodes); L.lom[l] = take(4 * nodes); }
    if (l >= 1 && keep && s.keep_debug) { L.rep[l] = take(4 * nodes); L.obs[l] = take(8 * nodes); }
    if (l >= 1 && l <= s.mat_top && s.keep_obs && L.obs[l] == kNone) L.obs[l] = take(8 * nodes);
  }
  L.bytes = off;
  return L;
}

int validate_plan_args(const vopp_model *m, int N, int D, int W, float eta, float gamma,
                       const float *pi_bar) {
  if (!m) return fail(VOPP_E_INVALID, "model is NULL");
  if (D < 0 || D > VOPP_MAX_DEPTH) return fail(VOPP_E_INVALID, "depth %d outside [0,%d]", D, VOPP_MAX_DEPTH);
  if (W < 1 || m->A * W > kMaxAW) return fail(VOPP_E_INVALID, "width %d invalid (A*W <= %d)", W, kMaxAW);
  if (N < 1 || N > VOPP_MAX_PARTICLES) return fail(VOPP_E_INVALID, "n_particles %d outside [1,%d]", N, VOPP_MAX_PARTICLES);
  // the leaf kernel stages one node's particle set in shared memory
  if (leaf_smem_bytes(m->desc.kind, N, m->A * W) > kLeafSmemLimit)
    return fail(VOPP_E_INVALID, "n_particles %d too large for the leaf kernel's node buffer", N);
  if (!(eta > 0.f) || !std::isfinite(eta)) return fail(VOPP_E_INVALID, "eta must be > 0");
  if (!(gamma > 0.f && gamma < 1.f)) return fail(VOPP_E_INVALID, "gamma must be in (0,1)");
  if (m->desc.branch_mode == VOPP_BRANCH_ENUMERATE) {
    const int nobs = m->host.n_obs;
    if (nobs <= 0 || W < nobs) return fail(VOPP_E_INVALID, "ENUMERATE needs a discrete model and width >= |O|");
  }
  if (pi_bar) {
    double s = 0.0;
    for (int a = 0; a < m->A; ++a) {
      if (!(pi_bar[a] >= 0.f) || !std::isfinite(pi_bar[a])) return fail(VOPP_E_INVALID, "pi_bar[%d] invalid", a);
      s += pi_bar[a];
    }
    if (!(s > 0.0)) return fail(VOPP_E_INVALID, "pi_bar sums to 0");
  }
  // tree size: nodes per level must stay inside 2^40 so that indices fit comfortably
  if ((double)D * std::log((double)m->A * W) > 40.0 * std::log(2.0))
    return fail(VOPP_E_INVALID, "tree too large");
  return VOPP_OK;
}

int ensure_arena(vopp_ctx *c, size_t bytes) {
  if (bytes <= c->arena_cap) return VOPP_OK;
  if (bytes > c->budget)
    return fail(VOPP_E_BUDGET, "plan needs %zu bytes, budget is %zu", bytes, c->budget);
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->arena) cudaFree(c->arena);
  c->arena = nullptr;
  c->arena_cap = 0;
  size_t want = std::min(c->budget, std::max(bytes, (size_t)(1.25 * (double)bytes)));
  want = align_up(want, 1 << 20);
  if (want > c->budget) want = bytes;
  if (cudaMalloc(&c->arena, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->arena = nullptr;
      return fail(VOPP_E_NOMEM, "cudaMalloc of %zu arena bytes failed", bytes);
    }
    want = bytes;
  }
  c->arena_cap = want;
  return VOPP_OK;
}

int ensure_meta(Slot &s, size_t bytes) {
  if (bytes <= s.meta_cap) return VOPP_OK;
  CUDA_TRY(cudaStreamSynchronize(s.stream));
  if (s.meta) cudaFree(s.meta);
  if (s.hmeta) cudaFreeHost(s.hmeta);
  s.meta = s.hmeta = nullptr;
  s.meta_cap = 0;
  const size_t want = align_up(std::max(bytes, (size_t)1 << 16) * 2, 1 << 16);
  if (cudaMalloc(&s.meta, want) != cudaSuccess) { cudaGetLastError(); return fail(VOPP_E_NOMEM, "meta alloc"); }
  if (cudaMallocHost(&s.hmeta, want) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s.meta);
    s.meta = nullptr;
    return fail(VOPP_E_NOMEM, "pinned meta alloc");
  }
  s.meta_cap = want;
  return VOPP_OK;
}

void free_slot(Slot &s) {
  if (s.meta) cudaFree(s.meta);
  if (s.hmeta) cudaFreeHost(s.hmeta);
  s.meta = s.hmeta = nullptr;
  s.meta_cap = 0;
}

// ---- timing -----------------------------------------------------------------------------
void timed_begin(vopp_ctx *c, int fam, TimedLaunch &t, int level = -1) {
  t.family = fam;
  t.level = level;
  t.a = t.b = nullptr;
  if (!c->timing) return;
  while (c->ev_pool.size() < c->ev_used + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  t.a = c->ev_pool[c->ev_used++];
  t.b = c->ev_pool[c->ev_used++];
  cudaEventRecord(t.a, c->stream);
}
void timed_end(vopp_ctx *c, TimedLaunch &t) {
  if (!c->timing) return;
  cudaEventRecord(t.b, c->stream);
  c->pending.push_back(t);
}
void timed_collect(vopp_ctx *c) {
  for (auto &t : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      c->fam_ms[t.family] += ms;
      c->fam_n[t.family] += 1;
      if (t.family == F_EXPAND && t.level >= 0 && t.level < kMaxDepth) {
        c->fam_ms[F_COUNT + t.level] += ms;
        c->fam_n[F_COUNT + t.level] += 1;
      }
    }
  }
  c->pending.clear();
  c->ev_used = 0;
}

// ---------------------------------------------------------------------------------------
// One launch sequence for a set of plans.
// ---------------------------------------------------------------------------------------
}  // namespace

// A tree kept on the device for subtree reuse: its memory (from the stream-ordered pool),
// its shape and layout, and the Philox key schedule its nodes were drawn with (key = seed,
// key level of its root, key node index of its root at that level).
struct KeptTree {
  char *mem = nullptr;
  size_t bytes = 0;
  PlanShape shape{};
  PlanLayout lay{};
  uint64_t seed = 0;
  int lvl_off = 0;
  unsigned long long root_idx = 0;
};

namespace {

struct Job {
  const vopp_model *model;
  PlanShape shape;
  PlanLayout lay;
  size_t arena_off;
  int first_expand = 0;     // levels 1..first_expand are already materialised (anytime)
  int psi_new_level = 0;    // anytime: levels >= this start from Psi_0
  const void *states;
  const float *weights;
  const float *log_weights;   // device log weights (agents)
  uint32_t ptr_flags;
  vopp_plan_params p;
  // subtree reuse
  vopp_agent *agent = nullptr;      // agent that keeps this plan's tree (own arena)
  char *own_arena = nullptr;        // the plan's memory when its tree is kept
  const KeptTree *reuse_src = nullptr;   // adopted subtree this plan continues
  int lvl_off = 0, reuse_root = 0;
  unsigned long long root_idx = 0;
};

struct StageBuild {
  int family;
  int level;
  int kind = -1;              // leaf and vectorised expansion stages: the model of every plan
  int vec_width = 0;          // vectorised expansions: particles per thread unit (0: generic)
  bool long_step = false;     // expansion stages: a CROWD plan (five Philox calls per step)
  std::vector<int> plans, levels;
  std::vector<long long> prefix;
  long long total = 0;
  int maxN = 0;
  size_t smem = 0;
  StageTable st{};
};

// CTAs of a persistent leaf launch: every SM filled to the kernel's occupancy.
int persistent_grid(vopp_ctx *c, int kind, size_t smem) {
  int per_sm = 0;
  if (leaf_occupancy(kind, c->leaf_threads, smem, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
  return per_sm * c->sm_count;
}

// Arena bytes of a batch; assigns each job its offset.
size_t place_jobs(std::vector<Job> &jobs) {
  size_t arena_bytes = 0;
  for (auto &j : jobs) {
    j.arena_off = arena_bytes;
    if (!j.agent) arena_bytes = align_up(arena_bytes + j.lay.bytes, 256);   // kept trees: own memory
  }
  return std::max<size_t>(arena_bytes, 256);
}

// Relative cost of one work item of a plan's leaf / expansion stage (for ordering).
double item_cost(const Job &j, bool leaf) {
  // relative cost of one particle-step (measured issue slots: NAV2D ~120, GRID ~85 less the
  // node build, CROWD ~690)
  const double per = (j.shape.kind == kNav) ? 2.0 : (j.shape.kind == kCrowd ? 11.0 : 1.0);
  return per * j.shape.N * (leaf ? (double)(j.shape.AW + 1) : 1.0);
}

// Plan indices of a stage, most expensive work items first (longest-processing-time order,
// so that the CTAs dispatched first carry the largest items).
std::vector<int> lpt_order(const std::vector<Job> &jobs, bool leaf) {
  std::vector<int> idx(jobs.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    return item_cost(jobs[x], leaf) > item_cost(jobs[y], leaf);
  });
  return idx;
}

// A device-to-device copy of a kept subtree's arrays into a plan's arena (src == nullptr:
// zero dst instead).
struct CopyOp {
  void *dst;
  const void *src;
  size_t bytes;
};

// Materialised levels a plan continuing a kept subtree takes from it (0: the root only).
int reuse_top(const vopp_ctx *c, const Job &j) {
  return c->reuse_copy ? std::min(j.reuse_src->shape.mat_top, j.shape.mat_top) : 0;
}

// The copies that put a kept subtree's levels 0..reuse_top into a plan's arena `base`:
// particle stores, branch statistics, observations and mean particles, and zeroed
// completion counters (the kernels that would have written them do not run).  level0:
// only level 0's (the root's particles and log weights); otherwise only levels >= 1.
void reuse_copies(const vopp_ctx *c, const Job &j, char *base, std::vector<CopyOp> &ops,
                  bool level0) {
  const KeptTree &t = *j.reuse_src;
  const PlanLayout &L = j.lay, &S = t.lay;
  const size_t N = (size_t)j.shape.N;
  const int top = reuse_top(c, j);
  auto add = [&](size_t d, size_t s, size_t bytes) {
    if (d != kNone && s != kNone) ops.push_back(CopyOp{base + d, t.mem + s, bytes});
  };
  for (int l = level0 ? 0 : 1; l <= (level0 ? 0 : top); ++l) {
    const size_t nodes = (size_t)ipow(j.shape.AW, l), n = nodes * N;
    add(L.px[l], S.px[l], 4 * n);
    add(L.py[l], S.py[l], 4 * n);
    add(L.ps[l], S.ps[l], 4 * n);
    add(L.pf[l], S.pf[l], 48 * n);
    add(L.plw[l], S.plw[l], 4 * n);
    if (l == 0) continue;
    add(L.rbar[l], S.rbar[l], 4 * nodes);
    add(L.lom[l], S.lom[l], 4 * nodes);
    add(L.obs[l], S.obs[l], 8 * nodes);
    add(L.rep[l], S.rep[l], 4 * nodes);
    add(L.mu[l], S.mu[l], 8 * nodes);
    if (L.cnt[l] != kNone) ops.push_back(CopyOp{base + L.cnt[l], nullptr, 4 * nodes});
  }
}

// Build the metadata block of a batch in the slot's pinned mirror, upload it and enqueue
// every launch and the device->host copy of the results on the slot's stream.  Nothing
// here waits for the device.
int enqueue_jobs(vopp_ctx *c, Slot &sl, char *arena, std::vector<Job> &jobs, bool timed,
                 GraphSet *graph) {
  const int n = (int)jobs.size();
  int rc = VOPP_OK;
  const std::vector<int> order_leaf = lpt_order(jobs, true), order_exp = lpt_order(jobs, false);

  // stages.  A plan whose first stage is the level-0 expansion lets that stage prepare its
  // root (one launch fewer on its critical path), unless it continues a kept subtree or its
  // root does not fit the expansion's shared memory.
  std::vector<StageBuild> stages;
  auto nodes = [](const Job &j, int l) { return (long long)ipow(j.shape.AW, l); };
  std::vector<char> fused(n, 0);
  for (int i = 0; i < n; ++i) {
    const Job &j = jobs[i];
    fused[i] = j.shape.mat_top >= 1 && j.first_expand == 0 && !j.reuse_root &&
               expand_fused_smem_bytes(j.shape.kind, j.shape.N) <= kLeafSmemLimit;
  }
  // A plan continuing a kept subtree with copies on (and no distance-softmax policy, whose
  // root mean a root preparation computes) needs no root preparation: its root is the kept
  // subtree's level 0 as it stands (a branch whose particles all have zero weight is never
  // adopted), its kernels read the stored levels from the subtree itself, and the copies that
  // make its own tree whole run off its critical path (a copy tail, below).
  std::vector<char> zc(n, 0);
  for (int i = 0; i < n; ++i) {
    const Job &j = jobs[i];
    zc[i] = j.reuse_src && c->reuse_copy && !(j.shape.pi_mode == kPiNavDist && !j.p.pi_bar);
  }
  {
    StageBuild s;
    s.family = F_ROOT;
    s.level = 0;
    for (int i = 0; i < n; ++i)
      if (!fused[i] && !zc[i]) { s.prefix.push_back((long long)s.plans.size()); s.plans.push_back(i); }
    s.prefix.push_back((long long)s.plans.size());
    s.total = (long long)s.plans.size();
    if (s.total) stages.push_back(s);
  }
  int max_mat = 0, maxD = 0;
  for (auto &j : jobs) { max_mat = std::max(max_mat, j.shape.mat_top); maxD = std::max(maxD, j.shape.D); }
  // Expansion stages, per level: vectorised launches for NAV2D, GRID and TOY2 plans (a fused
  // root preparation excepted), one per model and vector width (the widest of 4, 2, 1 that
  // divides the plan's N: a plan's particle-to-lane mapping, and so its rounding, depends
  // on nothing but the plan), and one generic launch for the rest (CROWD, the level-0
  // expansions that prepare their roots, levels of fewer than kExpandVecMinChildren nodes,
  // where one CTA per child is faster).  Work items are the level's children.
  for (int l = 0; l < max_mat; ++l) {
    auto takes = [&](int i) { return jobs[i].shape.mat_top > l && l >= jobs[i].first_expand; };
    auto vec_class = [&](int i) {   // (model, vector width), or (-1, 0) for the generic kernel
      const int kd = jobs[i].shape.kind, N = jobs[i].shape.N;
      // A small level is latency-bound: one CTA per child.  The choice goes by the level's
      // width in the full tree its Philox keys belong to (key level, not plan level), so that
      // a node is always built by the same kernel, and so rounded the same, whether a plan
      // builds it fresh or continues a kept subtree that holds it.
      long long w = 1;
      for (int t = 0; t <= l + jobs[i].lvl_off && w < kExpandVecMinChildren; ++t) w *= jobs[i].shape.AW;
      if (kd == kCrowd || (l == 0 && fused[i]) || w < kExpandVecMinChildren)
        return std::make_pair(-1, 0);
      return std::make_pair(kd, (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 1));
    };
    const std::pair<int, int> classes[] = {{-1, 0}, {kNav, 4}, {kNav, 2}, {kNav, 1},
                                           {kGrid, 4}, {kGrid, 2}, {kGrid, 1},
                                           {kToy, 4}, {kToy, 2}, {kToy, 1}};
    for (const auto &cls : classes) {
      const int kd = cls.first;
      StageBuild s;
      s.family = F_EXPAND;
      s.level = l;
      s.kind = kd;
      s.vec_width = cls.second;
      long long acc = 0;
      for (int i : order_exp) {
        if (!takes(i) || vec_class(i) != cls) continue;
        s.plans.push_back(i);
        s.levels.push_back(l);
        s.prefix.push_back(acc);
        acc += nodes(jobs[i], l + 1);
        s.maxN = std::max(s.maxN, jobs[i].shape.N);
        if (jobs[i].shape.kind == kCrowd) s.long_step = true;
        if (kd < 0)
          s.smem = std::max(s.smem, (l == 0 && fused[i])
                                        ? expand_fused_smem_bytes(jobs[i].shape.kind, jobs[i].shape.N)
                                        : expand_smem_bytes(jobs[i].shape.N));
      }
      if (!acc) continue;
      s.prefix.push_back(acc);
      s.total = acc;
      stages.push_back(s);
    }
  }
  // Leaf stage: one launch per model and shared-memory class (powers of two of the node
  // buffer), so that each model runs its own kernel and small-N plans are not held to the
  // occupancy of the largest node buffer.
  {
    auto leaf_class = [&](const Job &j) {
      const size_t b = leaf_smem_bytes(j.shape.kind, j.shape.N, j.shape.AW);
      int cls = 0;
      while (((size_t)1024 << cls) < b) ++cls;
      return std::make_pair(cls, j.shape.kind);
    };
    std::vector<std::pair<int, int>> classes;
    for (int i : order_leaf)
      if (jobs[i].shape.D >= 1) {
        const auto key = leaf_class(jobs[i]);
        if (std::find(classes.begin(), classes.end(), key) == classes.end()) classes.push_back(key);
      }
    std::sort(classes.begin(), classes.end(), [](const std::pair<int, int> &x,
                                                 const std::pair<int, int> &y) {
      return x.first != y.first ? x.first > y.first : x.second < y.second;
    });
    for (const auto &key : classes) {
      StageBuild s;
      s.family = F_LEAF;
      s.level = 0;
      s.kind = key.second;
      long long acc = 0;
      for (int i : order_leaf) {
        if (jobs[i].shape.D < 1 || leaf_class(jobs[i]) != key) continue;
        s.plans.push_back(i);
        s.prefix.push_back(acc);
        acc += nodes(jobs[i], jobs[i].shape.D - 1);
        s.smem = std::max(s.smem, leaf_smem_bytes(jobs[i].shape.kind, jobs[i].shape.N,
                                                  jobs[i].shape.AW));
      }
      s.prefix.push_back(acc);
      s.total = acc;
      if (acc) stages.push_back(s);
    }
  }
  // metadata block: [results n][descs n][stage tables][root copies]
  size_t off = 0;
  const size_t off_res = off; off = align_up(off + sizeof(DevResult) * n, 256);
  const size_t off_desc = off; off = align_up(off + sizeof(PlanDesc) * n, 256);
  std::vector<size_t> st_off(stages.size());
  for (size_t s = 0; s < stages.size(); ++s) {
    st_off[s] = off;
    const size_t k = stages[s].plans.size();
    off = align_up(off + 4 * k, 8);            // plan ids
    off = align_up(off + 8 * (k + 1), 8);      // prefix
    off = align_up(off + 4 * k, 8);            // levels
    off = align_up(off + 8, 256);              // work counter (persistent launches)
  }
  // copies of kept subtrees into the memory of the plans that continue them: their
  // descriptors travel in the metadata block, so that a recorded sequence can be replayed.
  // Levels >= 1 of every continued plan first (slices of them run as extra CTAs of the root
  // preparation launch), then each plan's level 0 (copied by its own root preparation CTA,
  // which reads it next); a continued plan always has a root preparation CTA.
  std::vector<CopyOp> copies;
  for (int i = 0; i < n; ++i) {
    const Job &j = jobs[i];
    if (!j.reuse_src) continue;
    char *base = j.own_arena ? j.own_arena : arena + j.arena_off;
    if (zc[i]) {   // every level's copies and the root's completion counter, in the tail
      reuse_copies(c, j, base, copies, true);
      if (j.shape.D >= 2 && j.lay.cnt[0] != kNone) copies.push_back(CopyOp{base + j.lay.cnt[0], nullptr, 4});
    }
    reuse_copies(c, j, base, copies, false);
  }
  const int n_rest = (int)copies.size();
  unsigned long long copy_most = 0;
  for (const CopyOp &op : copies) copy_most = std::max<unsigned long long>(copy_most, op.bytes);
  std::vector<int> copy0_first(n, 0), copy0_n(n, 0);
  bool copies_in_root = true;
  for (int i = 0; i < n; ++i) {
    const Job &j = jobs[i];
    if (!j.reuse_src || zc[i]) continue;
    copies_in_root = copies_in_root && !fused[i];
    copy0_first[i] = (int)copies.size();
    reuse_copies(c, j, j.own_arena ? j.own_arena : arena + j.arena_off, copies, true);
    copy0_n[i] = (int)copies.size() - copy0_first[i];
  }
  if (!copies_in_root)   // (not reached: a continued plan never fuses its root) one copy launch
    for (int i = 0; i < n; ++i) copy0_n[i] = 0;
  unsigned long long copy_most_all = copy_most;
  for (const CopyOp &op : copies) copy_most_all = std::max<unsigned long long>(copy_most_all, op.bytes);
  // where entries 0 .. n_rest - 1 run: in the root preparation launch when there is one, else
  // as the copy tail of the first expansion launch (both precede the leaves, whose climb
  // reads the zeroed counters), else in a copy launch of their own ahead of the leaves
  const bool has_root = !stages.empty() && stages[0].family == F_ROOT;
  int tail_stage = -1;
  if (n_rest > 0 && !has_root)
    for (size_t k = 0; k < stages.size(); ++k)
      if (stages[k].family == F_EXPAND) { tail_stage = (int)k; break; }
  const bool tail_separate = n_rest > 0 && !has_root && tail_stage < 0 && copies_in_root;
  const unsigned tail_slices = (unsigned)std::min<unsigned long long>(
      65535, std::max<unsigned long long>(1, (copy_most + (64ull << 10) - 1) / (64ull << 10)));
  const size_t off_copy = off;
  off = align_up(off + sizeof(CopyDesc) * copies.size(), 256);
  std::vector<size_t> root_off(n, kNone);
  for (int i = 0; i < n; ++i) {
    const Job &j = jobs[i];
    if (!(j.ptr_flags & VOPP_PTR_DEVICE) && j.states) {
      root_off[i] = off;
      const size_t sb = root_words(j.shape.kind) * 4 * (size_t)j.shape.N;
      const size_t wb = j.weights ? 4 * (size_t)j.shape.N : 0;
      off = align_up(off + sb + wb, 256);
    }
  }
  rc = ensure_meta(sl, off);
  if (rc) return rc;
  char *H = sl.hmeta, *Dm = sl.meta;
  std::memset(H, 0, off);
  sl.off_res = off_res;
  sl.off_desc = off_desc;
  sl.n = n;
  PlanDesc *hd = reinterpret_cast<PlanDesc *>(H + off_desc);
  const PlanDesc *dd = reinterpret_cast<const PlanDesc *>(Dm + off_desc);
  {
    CopyDesc *hc = reinterpret_cast<CopyDesc *>(H + off_copy);
    for (size_t q = 0; q < copies.size(); ++q)
      hc[q] = CopyDesc{copies[q].dst, copies[q].src, (unsigned long long)copies[q].bytes};
  }
  for (int i = 0; i < n; ++i) {
    const Job &j = jobs[i];
    const PlanShape &sh = j.shape;
    PlanDesc P;
    std::memset(&P, 0, sizeof P);
    P.kind = sh.kind; P.A = sh.A; P.W = sh.W; P.AW = sh.AW; P.N = sh.N; P.D = sh.D;
    P.branch_mode = j.model->desc.branch_mode;
    P.pi_mode = sh.pi_mode;
    P.h_zero = j.model->desc.h_zero;
    P.leaf_gen = sh.leaf_gen; P.keep_leaf = sh.keep_leaf; P.keep_debug = sh.keep_debug;
    P.fp64_root = c->fp64_root;
    P.eta = j.p.eta; P.inv_eta = 1.0f / j.p.eta; P.gamma = j.p.gamma;
    P.pi_temp = j.model->desc.pi_temp;
    // reference policy (uniform / fixed / caller override), normalised in double
    {
      double w[kMaxActions], s = 0.0;
      for (int a = 0; a < sh.A; ++a) {
        if (j.p.pi_bar) w[a] = j.p.pi_bar[a];
        else if (sh.pi_mode == kPiFixed) w[a] = j.model->desc.pi_fixed[a];
        else w[a] = 1.0;
        s += w[a];
      }
      for (int a = 0; a < sh.A; ++a) P.log_pi[a] = w[a] > 0.0 ? (float)std::log(w[a] / s) : -INFINITY;
      if (j.p.pi_bar && P.pi_mode == kPiNavDist) P.pi_mode = kPiFixed;
    }
    const double g = j.p.gamma;
    P.h_a0 = (float)(-1.0 / (1.0 - g));
    P.h_b0 = (float)((sh.kind == kCrowd ? 1000.0 : 100.0) + 1.0 / (1.0 - g));
    P.log2_gamma = (float)std::log2(g);
    P.key0 = (uint32_t)j.p.seed;
    P.key1 = (uint32_t)(j.p.seed >> 32);
    P.model = j.model->dev;
    P.lvl_off = j.lvl_off;
    P.reuse_root = j.reuse_root;
    P.root_fused = fused[i];
    P.copy0_first = copy0_first[i];
    P.copy0_n = copy0_n[i];
    for (int l = 0; l <= kMaxDepth; ++l)
      P.node_off[l] = (l <= sh.D) ? j.root_idx * ipow(sh.AW, l) : 0ull;
    char *base = j.own_arena ? j.own_arena : arena + j.arena_off;
    const PlanLayout &L = j.lay;
    auto fp = [&](size_t o) { return o == kNone ? nullptr : reinterpret_cast<float *>(base + o); };
    auto ip = [&](size_t o) { return o == kNone ? nullptr : reinterpret_cast<int *>(base + o); };
    for (int l = 0; l < kMaxDepth; ++l) {
      P.px[l] = fp(L.px[l]); P.py[l] = fp(L.py[l]); P.plw[l] = fp(L.plw[l]); P.ps[l] = ip(L.ps[l]);
      P.pf[l] = fp(L.pf[l]);
      P.Q[l] = fp(L.Q[l]); P.mu[l] = fp(L.mu[l]);
      P.cnt[l] = L.cnt[l] == kNone ? nullptr : reinterpret_cast<unsigned int *>(base + L.cnt[l]);
      P.psi[l] = fp(L.psi[l]);
    }
    P.psi_new_level = j.psi_new_level;
    for (int l = 0; l <= kMaxDepth; ++l) {
      P.rbar[l] = fp(L.rbar[l]); P.lom[l] = fp(L.lom[l]); P.V[l] = fp(L.V[l]);
      P.rep[l] = ip(L.rep[l]); P.obs[l] = fp(L.obs[l]);
    }
    if (zc[i]) {   // the stored levels are read from the kept subtree (copied for the tree later)
      const KeptTree &t = *j.reuse_src;
      const PlanLayout &S = t.lay;
      auto sfp = [&](size_t o, float *own) { return o == kNone ? own : reinterpret_cast<float *>(t.mem + o); };
      auto sip = [&](size_t o, int *own) { return o == kNone ? own : reinterpret_cast<int *>(t.mem + o); };
      const int top = reuse_top(c, j);
      for (int l = 0; l <= top; ++l) {
        P.px[l] = sfp(S.px[l], P.px[l]); P.py[l] = sfp(S.py[l], P.py[l]);
        P.plw[l] = sfp(S.plw[l], P.plw[l]); P.ps[l] = sip(S.ps[l], P.ps[l]);
        P.pf[l] = sfp(S.pf[l], P.pf[l]);
        if (l == 0) continue;
        P.rbar[l] = sfp(S.rbar[l], P.rbar[l]); P.lom[l] = sfp(S.lom[l], P.lom[l]);
        P.obs[l] = sfp(S.obs[l], P.obs[l]); P.rep[l] = sip(S.rep[l], P.rep[l]);
      }
    }
    P.result = reinterpret_cast<DevResult *>(Dm + off_res) + i;
    // root input
    if (j.log_weights) {
      P.root_lw = j.log_weights;
    }
    // root states: NAV2D rows x, y; GRID / TOY2 one row s; CROWD rows x, y, 12 people, flags
    auto set_root = [&](const char *base) {
      if (sh.kind == kNav || sh.kind == kCrowd) {
        P.root_x = reinterpret_cast<const float *>(base);
        P.root_y = P.root_x + sh.N;
      }
      if (sh.kind == kCrowd) {
        P.root_pf = P.root_x + 2 * (size_t)sh.N;
        P.root_s = reinterpret_cast<const int *>(P.root_x + 14 * (size_t)sh.N);
      } else if (sh.kind != kNav) {
        P.root_s = reinterpret_cast<const int *>(base);
      }
    };
    if (j.ptr_flags & VOPP_PTR_DEVICE || !j.states) {
      set_root(static_cast<const char *>(j.states));
      P.root_w = j.weights;
    } else {
      char *hb = H + root_off[i];
      const char *db = Dm + root_off[i];
      const size_t sb = root_words(sh.kind) * 4 * (size_t)sh.N;
      std::memcpy(hb, j.states, sb);
      set_root(db);
      if (j.weights) {
        std::memcpy(hb + sb, j.weights, 4 * (size_t)sh.N);
        P.root_w = reinterpret_cast<const float *>(db + sb);
      }
    }
    hd[i] = P;
  }
  for (size_t s = 0; s < stages.size(); ++s) {
    StageBuild &sb = stages[s];
    const size_t k = sb.plans.size();
    size_t o = st_off[s];
    int *hp = reinterpret_cast<int *>(H + o);
    for (size_t i = 0; i < k; ++i) hp[i] = sb.plans[i];
    sb.st.plan = reinterpret_cast<const int *>(Dm + o);
    o = align_up(o + 4 * k, 8);
    long long *hq = reinterpret_cast<long long *>(H + o);
    for (size_t i = 0; i <= k; ++i) hq[i] = sb.prefix[i];
    sb.st.prefix = reinterpret_cast<const long long *>(Dm + o);
    o = align_up(o + 8 * (k + 1), 8);
    if (!sb.levels.empty()) {
      int *hl = reinterpret_cast<int *>(H + o);
      for (size_t i = 0; i < k; ++i) hl[i] = sb.levels[i];
      sb.st.levels = reinterpret_cast<const int *>(Dm + o);
    } else {
      sb.st.levels = nullptr;
    }
    o = align_up(o + 4 * k, 8);
    sb.st.counter = reinterpret_cast<unsigned long long *>(Dm + o);   // zeroed by the upload
    sb.st.n_plans = (int)k;
    sb.st.level = sb.level;
  }
  cudaStream_t stream = sl.stream;
  c->h2d_bytes += off;
  c->d2h_bytes += sizeof(DevResult) * n;
  c->launches += stages.size();
  // launch shapes (computed before any capture)
  std::vector<long long> grids(stages.size());
  for (size_t k = 0; k < stages.size(); ++k) {
    StageBuild &sb = stages[k];
    if (sb.family == F_LEAF) {
      const bool pers = (c->leaf_persistent == 2) ? (sb.kind == kGrid || sb.kind == kToy)
                                                  : c->leaf_persistent != 0;
      if (!pers) sb.st.counter = nullptr;
      grids[k] = pers ? persistent_grid(c, sb.kind, sb.smem) : std::min<long long>(sb.total, c->grid_cap);
    } else if (sb.family == F_EXPAND) {
      const long long per = sb.vec_width ? kExpandVecChildrenPerCta : 1;
      grids[k] = std::min<long long>((sb.total + per - 1) / per, c->grid_cap);
      if ((int)k == tail_stage) {   // the copy tail of continued subtrees
        sb.st.copies = Dm + off_copy;
        sb.st.n_copies = n_rest;
        sb.st.copy_slices = tail_slices;
        sb.st.work_grid = (unsigned)grids[k];
        grids[k] += (long long)n_rest * tail_slices;
      }
    } else {
      grids[k] = sb.st.n_plans;
    }
  }
  auto record = [&](cudaStream_t stream) -> int {
    CUDA_TRY(cudaMemcpyAsync(Dm, H, off, cudaMemcpyHostToDevice, stream));
    if (!copies.empty() && !copies_in_root)   // one launch for every copy, after the upload
      CUDA_TRY(launch_copy_table(reinterpret_cast<const CopyDesc *>(Dm + off_copy), (int)copies.size(),
                                 copy_most_all, stream));
    if (tail_separate)   // continued subtrees' copies with no launch to ride in before the leaves
      CUDA_TRY(launch_copy_table(reinterpret_cast<const CopyDesc *>(Dm + off_copy), n_rest, copy_most,
                                 stream));
    for (size_t k = 0; k < stages.size(); ++k) {
      StageBuild &sb = stages[k];
      TimedLaunch tl;
      vopp::NvtxRange nvtx_range(sb.family == F_ROOT ? "k_root_prep" :
                                 (sb.family == F_EXPAND ? "k_expand" : "k_leaf"));
      if (timed) timed_begin(c, sb.family, tl, sb.family == F_EXPAND ? sb.level : -1);
      cudaError_t e = cudaSuccess;
      switch (sb.family) {
        case F_ROOT:
          e = (copies.empty() || !copies_in_root)
                  ? launch_root_prep(dd, sb.st, stream)
                  : launch_root_prep_copy(dd, sb.st, reinterpret_cast<const CopyDesc *>(Dm + off_copy),
                                          n_rest, copy_most, stream);
          break;
        case F_EXPAND:
          // a level of long steps with at most one CTA per SM takes wider CTAs (fewer
          // particles per thread on its critical path; measured faster for CROWD only)
          if (sb.vec_width)
            e = launch_expand_vec(sb.kind, sb.vec_width, dd, sb.st, sb.total, grids[k], stream);
          else
            e = launch_expand(dd, sb.st, sb.total, sb.smem, grids[k],
                              sb.long_step && grids[k] <= c->sm_count, stream);
          break;
        case F_LEAF: e = launch_leaf(sb.kind, dd, sb.st, sb.total, sb.smem, c->leaf_threads, grids[k], stream); break;
      }
      if (timed) timed_end(c, tl);
      if (e != cudaSuccess) return fail(VOPP_E_CUDA, "launch failed: %s", cudaGetErrorString(e));
    }
    CUDA_TRY(cudaMemcpyAsync(H + off_res, Dm + off_res, sizeof(DevResult) * n, cudaMemcpyDeviceToHost,
                             stream));
    return VOPP_OK;
  };
  if (!graph || timed) return record(stream);

  // signature of everything the recorded operations depend on
  std::vector<unsigned char> sig;
  auto put = [&](const void *p, size_t b) {
    const unsigned char *q = static_cast<const unsigned char *>(p);
    sig.insert(sig.end(), q, q + b);
  };
  const void *ptrs[2] = {Dm, H};
  put(ptrs, sizeof ptrs);
  put(&off, sizeof off);
  put(&off_res, sizeof off_res);
  put(&off_copy, sizeof off_copy);
  const size_t n_copies = copies.size();
  put(&n_copies, sizeof n_copies);
  put(&copy_most, sizeof copy_most);
  put(&n_rest, sizeof n_rest);
  put(&copies_in_root, sizeof copies_in_root);
  put(&tail_stage, sizeof tail_stage);
  put(&tail_separate, sizeof tail_separate);
  put(&n, sizeof n);
  put(&c->leaf_threads, sizeof c->leaf_threads);
  for (size_t k = 0; k < stages.size(); ++k) {
    const StageBuild &sb = stages[k];
    put(&sb.family, sizeof sb.family);
    put(&sb.kind, sizeof sb.kind);
    put(&sb.long_step, sizeof sb.long_step);
    put(&sb.vec_width, sizeof sb.vec_width);
    put(&sb.total, sizeof sb.total);
    put(&sb.smem, sizeof sb.smem);
    put(&sb.maxN, sizeof sb.maxN);
    put(&sb.st, sizeof sb.st);
    put(&grids[k], sizeof grids[k]);
  }
  const std::string key(sig.begin(), sig.end());
  auto it = graph->execs.find(key);
  if (it != graph->execs.end()) {
    CUDA_TRY(cudaGraphLaunch(it->second, stream));
    return VOPP_OK;
  }
  // a sequence not seen before runs directly; then, while the device works on it, it is
  // recorded and instantiated for the next time (a failed capture only means no replay)
  const int rc1 = record(stream);
  if (rc1 != VOPP_OK) return rc1;
  if (!graph->capture && cudaStreamCreateWithFlags(&graph->capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return VOPP_OK;
  }
  if (cudaStreamBeginCapture(graph->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return VOPP_OK;
  }
  const int rc2 = record(graph->capture);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(graph->capture, &g);
  cudaGraphExec_t exec = nullptr;
  if (rc2 == VOPP_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
    if (graph->order.size() >= GraphSet::kMaxGraphs) {
      auto old = graph->execs.find(graph->order.front());
      if (old != graph->execs.end()) {
        cudaGraphExecDestroy(old->second);
        graph->execs.erase(old);
      }
      graph->order.pop_front();
    }
    graph->execs.emplace(key, exec);
    graph->order.push_back(key);
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return VOPP_OK;
}

// Fill the results of a batch whose launches have completed on the slot's stream.
int collect_results(vopp_ctx *c, const Slot &sl, const std::vector<Job> &jobs,
                    vopp_plan_result *outs, int *statuses, bool remember) {
  const int n = (int)jobs.size();
  const PlanDesc *hd = reinterpret_cast<const PlanDesc *>(sl.hmeta + sl.off_desc);
  if (remember) {
    c->last_desc.assign(hd, hd + n);
    c->last_ok.assign(n, 1);
    // a plan that read its stored levels from a kept subtree has them in its own memory too
    // (the copy tail): the tree record points there, the subtree being released later
    for (int i = 0; i < n; ++i) {
      const Job &j = jobs[i];
      if (!j.reuse_src || !j.own_arena) continue;
      PlanDesc &D = c->last_desc[i];
      const PlanLayout &L = j.lay;
      auto fp = [&](size_t o, float *cur) { return o == kNone ? cur : reinterpret_cast<float *>(j.own_arena + o); };
      auto ip = [&](size_t o, int *cur) { return o == kNone ? cur : reinterpret_cast<int *>(j.own_arena + o); };
      const int top = reuse_top(c, j);
      for (int l = 0; l <= top; ++l) {
        D.px[l] = fp(L.px[l], D.px[l]); D.py[l] = fp(L.py[l], D.py[l]);
        D.plw[l] = fp(L.plw[l], D.plw[l]); D.ps[l] = ip(L.ps[l], D.ps[l]);
        D.pf[l] = fp(L.pf[l], D.pf[l]);
        if (l == 0) continue;
        D.rbar[l] = fp(L.rbar[l], D.rbar[l]); D.lom[l] = fp(L.lom[l], D.lom[l]);
        D.obs[l] = fp(L.obs[l], D.obs[l]); D.rep[l] = ip(L.rep[l], D.rep[l]);
      }
    }
  }
  const DevResult *hr = reinterpret_cast<const DevResult *>(sl.hmeta + sl.off_res);
  int first_err = VOPP_OK;
  for (int i = 0; i < n; ++i) {
    const Job &j = jobs[i];
    vopp_plan_result &o = outs[i];
    std::memset(&o, 0, sizeof o);
    int st = VOPP_OK;
    if (hr[i].status & kStatusDegenerateRoot) {
      st = VOPP_E_DEGENERATE;
      o.action = -1;
      if (remember) c->last_ok[i] = 0;
    } else {
      o.action = hr[i].action;
      o.v_root = hr[i].v_root;
      for (int a = 0; a < j.shape.A; ++a) { o.q[a] = hr[i].q[a]; o.policy[a] = hr[i].policy[a]; }
    }
    o.flags = hr[i].flags | (hr[i].degenerate ? VOPP_FLAG_DEGENERATE_BRANCH : 0u);
    o.degenerate_actions = hr[i].degenerate;
    if (j.reuse_src) {
      o.flags |= VOPP_FLAG_REUSED;
      o.reused_levels = (uint32_t)reuse_top(c, j);
    }
    unsigned long long steps = 0, nodes_total = 1;
    for (int l = 1; l <= j.shape.D; ++l) {
      steps += ipow(j.shape.AW, l) * (unsigned long long)j.shape.N;
      nodes_total += ipow(j.shape.AW, l);
    }
    o.particle_steps = steps;
    o.nodes = nodes_total;
    if (statuses) statuses[i] = st;
    if (st && !first_err) first_err = st;
  }
  if (first_err == VOPP_E_DEGENERATE) fail(VOPP_E_DEGENERATE, "root belief has zero total weight");
  return first_err;
}

// ---- subtree reuse ----------------------------------------------------------------------
void free_kept(KeptTree *&t, cudaStream_t s) {
  if (!t) return;
  if (t->mem) cudaFreeAsync(t->mem, s);
  delete t;
  t = nullptr;
}

// The Philox counter of every node of a depth-D tree rooted at key level lvl_off, key node
// root_idx fits: levels below 256 (8 bits) and node indices root_idx (A W)^l + n < 2^64.
bool keys_fit(int lvl_off, unsigned long long root_idx, int AW, int D) {
  if (lvl_off + D > 255) return false;
  unsigned __int128 span = 1;
  for (int l = 0; l < D; ++l) span *= (unsigned)AW;
  return ((unsigned __int128)root_idx + 1) * span <= ((unsigned __int128)1 << 64);
}

// An agent plan with subtree reuse on keeps its tree (own memory, observations of every
// materialised level), and continues the adopted subtree when the agent has one that fits
// (same width, keys within range): its keys, its root as it stands, its levels.
void attach_reuse(vopp_agent *g, Job &j) {
  j.agent = g;
  j.shape.keep_obs = 1;
  const KeptTree *sb = g->sub;
  if (sb && sb->shape.W == j.shape.W && sb->shape.N == j.shape.N &&
      keys_fit(sb->lvl_off, sb->root_idx, j.shape.AW, j.shape.D)) {
    j.reuse_src = sb;
    j.lvl_off = sb->lvl_off;
    j.root_idx = sb->root_idx;
    j.reuse_root = 1;
    j.p.seed = sb->seed;
    j.first_expand = j.model->ctx->reuse_copy ? std::min(sb->shape.mat_top, j.shape.mat_top) : 0;
  }
  j.lay = make_layout(j.shape);
}

// Release an agent's kept tree, its memory becoming the agent's spare (the larger of the two
// is kept) once the work enqueued on s so far -- the last that read it -- has completed.
void release_kept(vopp_agent *g, KeptTree *&t, cudaStream_t s) {
  if (t && t->mem && (!g->spare || t->bytes > g->spare_bytes)) {
    if (g->spare_ev || cudaEventCreateWithFlags(&g->spare_ev, cudaEventDisableTiming) == cudaSuccess) {
      if (cudaEventRecord(g->spare_ev, s) == cudaSuccess) {
        if (g->spare) cudaFreeAsync(g->spare, s);
        g->spare = t->mem;
        g->spare_bytes = t->bytes;
        t->mem = nullptr;
      }
    }
    cudaGetLastError();
  }
  free_kept(t, s);
}

// Memory of at least `bytes` for an agent's plan from its spare, or null (the caller
// allocates).
char *take_spare(vopp_agent *g, size_t bytes) {
  if (!g->spare || g->spare_bytes < bytes) return nullptr;
  const cudaError_t q = cudaEventQuery(g->spare_ev);
  if (q != cudaSuccess) {
    if (q != cudaErrorNotReady) cudaGetLastError();
    return nullptr;
  }
  char *p = g->spare;
  g->spare = nullptr;
  g->spare_bytes = 0;
  return p;
}

// After an agent's plan: its tree replaces the agent's kept tree (or is released if the
// plan failed).
void keep_tree(vopp_agent *g, Job &j, bool ok, cudaStream_t s) {
  release_kept(g, g->tree, s);
  if (!ok || !j.own_arena) {
    if (j.own_arena) cudaFreeAsync(j.own_arena, s);
    j.own_arena = nullptr;
    return;
  }
  KeptTree *t = new KeptTree;
  t->mem = j.own_arena;
  t->bytes = j.lay.bytes;
  t->shape = j.shape;
  t->lay = j.lay;
  t->seed = j.p.seed;
  t->lvl_off = j.lvl_off;
  t->root_idx = j.root_idx;
  g->tree = t;
  j.own_arena = nullptr;
}

// Adopt child `slot` (= a W + k) of the kept tree's root: its particle set becomes the
// agent's belief, and its materialised subtree (levels 1..mat_top of the tree, the child's
// nodes, contiguous at every level) is kept where it is: the subtree is a view into the
// tree's memory, which it takes over (level l of the subtree is the child's part of the
// tree's level l + 1), keyed as it was.  Only the belief is copied.
int adopt_subtree(vopp_agent *g, int slot, cudaStream_t s) {
  KeptTree &t = *g->tree;
  const int AW = t.shape.AW;
  const size_t N = (size_t)t.shape.N;
  PlanShape sh = t.shape;
  sh.D = t.shape.D - 1;
  sh.mat_top = t.shape.mat_top - 1;
  sh.keep_leaf = sh.keep_debug = 0;
  sh.keep_obs = 1;
  KeptTree *sb = new (std::nothrow) KeptTree;
  if (!sb) return fail(VOPP_E_NOMEM, "subtree alloc");
  sb->shape = sh;
  sb->seed = t.seed;
  sb->lvl_off = t.lvl_off + 1;
  sb->root_idx = t.root_idx * (unsigned long long)AW + (unsigned long long)slot;
  const PlanLayout &S = t.lay;
  PlanLayout &L = sb->lay;
  size_t *fields[] = {L.px, L.py, L.plw, L.ps, L.pf, L.Q, L.mu, L.cnt, L.psi};
  for (size_t *f : fields)
    for (int l = 0; l < kMaxDepth; ++l) f[l] = kNone;
  size_t *fields1[] = {L.rbar, L.lom, L.V, L.rep, L.obs};
  for (size_t *f : fields1)
    for (int l = 0; l <= kMaxDepth; ++l) f[l] = kNone;
  L.bytes = t.lay.bytes;
  auto at = [](size_t base, size_t off) { return base == kNone ? kNone : base + off; };
  for (int l = 0; l <= sh.mat_top; ++l) {
    const size_t nodes = (size_t)ipow(AW, l), first = (size_t)slot * nodes;   // first node there
    L.px[l] = at(S.px[l + 1], 4 * first * N);
    L.py[l] = at(S.py[l + 1], 4 * first * N);
    L.ps[l] = at(S.ps[l + 1], 4 * first * N);
    L.pf[l] = at(S.pf[l + 1], 48 * first * N);
    L.plw[l] = at(S.plw[l + 1], 4 * first * N);
    if (l == 0) continue;
    L.rbar[l] = at(S.rbar[l + 1], 4 * first);
    L.lom[l] = at(S.lom[l + 1], 4 * first);
    L.obs[l] = at(S.obs[l + 1], 8 * first);
    L.mu[l] = at(S.mu[l + 1], 8 * first);
  }
  // the agent's belief: the adopted node's particles in the agent's row layout
  cudaError_t e = cudaSuccess;
  std::vector<CopyOp> ops;
  auto cpa = [&](void *d, size_t src, size_t elem_bytes, size_t rows) {
    if (src != kNone) ops.push_back(CopyOp{d, t.mem + src + (size_t)slot * N * elem_bytes, rows * 4 * N});
  };
  const int kind = t.shape.kind;
  if (kind == kNav || kind == kCrowd) { cpa(g->xy, S.px[1], 4, 1); cpa(g->xy + N, S.py[1], 4, 1); }
  if (kind == kCrowd) cpa(g->pf, S.pf[1], 48, 12);
  if (kind != kNav) cpa(g->s, S.ps[1], 4, 1);
  cpa(g->lw, S.plw[1], 4, 1);
  for (size_t b = 0; e == cudaSuccess && b < ops.size(); b += kMaxCopyOps) {
    CopyList cl;
    cl.n = (int)std::min<size_t>(kMaxCopyOps, ops.size() - b);
    for (int q = 0; q < cl.n; ++q) {
      cl.dst[q] = ops[b + q].dst;
      cl.src[q] = ops[b + q].src;
      cl.bytes[q] = ops[b + q].bytes;
    }
    e = launch_copy_list(cl, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete sb;
    return fail(VOPP_E_CUDA, "belief copy: %s", cudaGetErrorString(e));
  }
  sb->mem = t.mem;        // the subtree takes the tree's memory over
  sb->bytes = t.bytes;
  t.mem = nullptr;
  release_kept(g, g->sub, s);
  g->sub = sb;
  return VOPP_OK;
}

// The kept tree's branch (action, k) whose sampled observation equals obs (lowest k), as
// slot action W + k, or -1.  Only a tree whose level 1 is materialised can be adopted.
int matching_branch(vopp_agent *g, int action, const float *obs_f, int obs_i, cudaStream_t s) {
  const KeptTree *t = g->tree;
  if (!t || t->shape.mat_top < 1 || t->lay.obs[1] == kNone) return -1;
  const int W = t->shape.W;
  // the action's branch observations and branch weights (a branch whose particles all have
  // zero weight, log omega = -inf, is never adopted: its belief would be degenerate)
  std::vector<float> ob(2 * (size_t)W), lo((size_t)W, 0.0f);
  if (cudaMemcpyAsync(ob.data(), t->mem + t->lay.obs[1] + 8 * (size_t)action * W, 8 * (size_t)W,
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      (t->lay.lom[1] != kNone &&
       cudaMemcpyAsync(lo.data(), t->mem + t->lay.lom[1] + 4 * (size_t)action * W, 4 * (size_t)W,
                       cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  for (int k = 0; k < W; ++k) {
    const bool eq = (t->shape.kind == kNav) ? (ob[2 * k] == obs_f[0] && ob[2 * k + 1] == obs_f[1])
                                            : ((int)ob[2 * k] == obs_i);
    if (eq) return (lo[k] > -INFINITY) ? action * W + k : -1;
  }
  return -1;
}

// Calls that use the context's arena, stream order or last-plan record wait for a plan
// that vopp_plan_submit left pending to be collected first.
int check_not_pending(const vopp_ctx *c) {
  return c->plan_pending ? fail(VOPP_E_BUSY, "a submitted plan is pending: call vopp_plan_finish")
                         : VOPP_OK;
}

int run_jobs(vopp_ctx *c, std::vector<Job> &jobs, vopp_plan_result *outs, int *statuses) {
  if (const int busy = check_not_pending(c)) return busy;
  int rc = ensure_arena(c, place_jobs(jobs));
  if (rc) return rc;
  c->slot.stream = c->stream;
  rc = enqueue_jobs(c, c->slot, c->arena, jobs, c->timing, c->use_graphs ? &c->graph : nullptr);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  timed_collect(c);
  return collect_results(c, c->slot, jobs, outs, statuses, true);
}

// GRID states as the kernels take them: bits 0-7 rocks, x (bits 8-11) in 0..11 with 11 =
// exited, y (bits 12-15) in 0..10, bit 16 terminal, bits 17-31 clear.
int check_grid_states(const vopp_model *m, const void *states, int n) {
  if (m->desc.kind != VOPP_GRID) return VOPP_OK;
  const int32_t *s = static_cast<const int32_t *>(states);
  for (int i = 0; i < n; ++i) {
    const int32_t v = s[i];
    if ((v & ~0x1FFFF) != 0 || ((v >> 8) & 0xF) > 11 || ((v >> 12) & 0xF) > 10)
      return fail(VOPP_E_INVALID, "grid state %d (0x%x) is not a packed state", i, (unsigned)v);
  }
  return VOPP_OK;
}

int make_job(vopp_ctx *c, vopp_model *m, const void *states, const float *weights, int N,
             const vopp_plan_params &p, uint32_t ptr_flags, Job &j) {
  int rc = validate_plan_args(m, N, p.depth, p.width, p.eta, p.gamma, p.pi_bar);
  if (rc) return rc;
  if (!states) return fail(VOPP_E_INVALID, "root_states is NULL");
  if (!(ptr_flags & VOPP_PTR_DEVICE) && (rc = check_grid_states(m, states, N))) return rc;
  if (weights && !(ptr_flags & VOPP_PTR_DEVICE)) {
    double s = 0.0;
    for (int i = 0; i < N; ++i) {
      if (!(weights[i] >= 0.f) || !std::isfinite(weights[i])) return fail(VOPP_E_INVALID, "weight %d invalid", i);
      s += weights[i];
    }
    if (!(s > 0.0)) return fail(VOPP_E_DEGENERATE, "root weights sum to 0");
  }
  j.model = m;
  j.shape = make_shape(m, N, p.depth, p.width, c);
  j.lay = make_layout(j.shape);
  j.states = states;
  j.weights = weights;
  j.log_weights = nullptr;
  j.ptr_flags = ptr_flags;
  j.p = p;
  return VOPP_OK;
}

// Anytime planning loop (Alg. 1): iterations k = 1, 2, ... each search the full-width tree
// of depth k with the plan's keys (so every node keeps its particle set from one iteration
// to the next) and back it up with the preference update of Eq. 3 on preferences that
// persist in the arena.  Iteration k materialises only the one level it adds above the leaf
// kernel's node level; the others are already in place.  The next iteration starts while
// the elapsed time is below budget_s (<= 0: no time limit) and k < the maximum depth.
int run_anytime(vopp_ctx *c, Job &base, double budget_s, vopp_plan_result *out, int *depth_out) {
  if (const int busy = check_not_pending(c)) return busy;
  const int K = base.p.depth;
  if (K < 1) return fail(VOPP_E_INVALID, "anytime planning needs a maximum depth >= 1");
  if (!(budget_s == budget_s)) return fail(VOPP_E_INVALID, "budget is NaN");
  base.lay = make_layout(base.shape, true);     // the depth-K arrays, shared by every iteration
  std::vector<Job> jobs(1, base);
  int rc = ensure_arena(c, place_jobs(jobs));
  if (rc) return rc;
  c->slot.stream = c->stream;
  const auto t0 = std::chrono::steady_clock::now();
  const unsigned long long N = (unsigned long long)base.shape.N, AW = base.shape.AW;
  unsigned long long steps = 0, nodes = 1;
  int prev_mat = 0, done = 0;
  vopp_plan_result res;
  for (int k = 1; k <= K; ++k) {
    Job &j = jobs[0];
    j.shape = make_shape(j.model, base.shape.N, k, base.shape.W, c);
    j.first_expand = prev_mat;
    j.psi_new_level = k - 1;
    j.p.depth = k;
    rc = enqueue_jobs(c, c->slot, c->arena, jobs, c->timing, nullptr);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    timed_collect(c);
    rc = collect_results(c, c->slot, jobs, &res, nullptr, true);
    if (rc) return rc;
    // particle-steps simulated by this iteration: the newly materialised levels, the node
    // level the leaf kernel builds in shared memory, and the leaves
    for (int l = prev_mat + 1; l <= j.shape.mat_top; ++l) steps += ipow(AW, l) * N;
    if (j.shape.leaf_gen) steps += ipow(AW, k - 1) * N;
    steps += ipow(AW, k) * N;
    nodes += ipow(AW, k);
    prev_mat = j.shape.mat_top;
    done = k;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (budget_s > 0.0 && el >= budget_s) break;
  }
  res.particle_steps = steps;
  res.nodes = nodes;
  *out = res;
  if (depth_out) *depth_out = done;
  return VOPP_OK;
}

void fill_grid_tables(DevModel &d, const vopp_model_desc &m) {
  for (int c = 0; c < 121; ++c) d.rock_at[c] = -1;
  for (int r = 0; r < 8; ++r) {
    d.rock_x[r] = m.rock_x[r];
    d.rock_y[r] = m.rock_y[r];
    d.rock_at[m.rock_x[r] + 11 * m.rock_y[r]] = r;
  }
  for (int d2 = 0; d2 < kGridD2; ++d2) {
    const double acc = 0.5 + 0.5 * std::exp(-std::sqrt((double)d2) / 4.0);
    d.thr[d2] = (unsigned long long)std::floor(acc * 4294967296.0);
    d.lacc[d2] = (float)std::log(acc);
    d.l1macc[d2] = (acc < 1.0) ? (float)std::log(1.0 - acc) : -INFINITY;
    d.lacc2[d2] = (float)std::log2(acc);
    d.l1macc2[d2] = (acc < 1.0) ? (float)std::log2(1.0 - acc) : -INFINITY;
    d.pz[d2] = (float)acc;
    d.pz[kGridD2 + d2] = (float)(1.0 - acc);
  }
}

}  // namespace

// Accessors used by entry points defined in other translation units.
namespace vopp {
const DevModel *model_device_tables(const vopp_model *m) { return m->dev; }
int model_kind(const vopp_model *m) { return m->desc.kind; }
int model_device(const vopp_model *m) { return m->ctx->device; }
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }
const vopp_model_desc &model_desc(const vopp_model *m) { return m->desc; }
vopp_ctx *model_ctx(const vopp_model *m) { return m->ctx; }
cudaStream_t model_stream(const vopp_model *m) { return m->ctx->stream; }
cudaStream_t ctx_stream(const vopp_ctx *c) { return c->stream; }
EpisodeStore *&ctx_episode_store(vopp_ctx *c) { return c->episodes; }
}  // namespace vopp

// ---------------------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------------------
extern "C" {

const char *vopp_last_error(void) { return g_err.c_str(); }
const char *vopp_version(void) { return "vopp-b300 0.1 (sm_103a)"; }

int vopp_ctx_create(int device, size_t hbm_budget_bytes, uintptr_t cuda_stream, vopp_ctx **out) {
  if (!out) return fail(VOPP_E_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(VOPP_E_INVALID, "device %d of %d", device, ndev);
  CUDA_TRY(cudaSetDevice(device));
  vopp_ctx *c = new (std::nothrow) vopp_ctx;
  if (!c) return fail(VOPP_E_NOMEM, "ctx alloc");
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete c; return fail(VOPP_E_CUDA, "cudaMemGetInfo"); }
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)fr);
  c->slot.stream = c->stream;
  if (init_kernel_attributes() != cudaSuccess) { delete c; return fail(VOPP_E_CUDA, "kernel attributes"); }
  {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    uint64_t keep = ~0ull;   // never return memory to the driver between allocations
    int no = 0;              // reuse memory only when its free has completed: no cross-stream waits
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no) != cudaSuccess) {
      cudaGetLastError();
      if (c->pool) cudaMemPoolDestroy(c->pool);
      delete c;
      return fail(VOPP_E_CUDA, "memory pool");
    }
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
    c->sm_count = sms;
  *out = c;
  return VOPP_OK;
}

void vopp_ctx_destroy(vopp_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  c->graph.release();
  free_episode_store(c->episodes);
  if (c->arena) cudaFree(c->arena);
  free_slot(c->slot);
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->pool) cudaMemPoolDestroy(c->pool);   // released once its last allocation is freed
  delete c;
}

int vopp_ctx_set_tree_detail(vopp_ctx *c, int detail) {
  if (!c || (detail != VOPP_TREE_MINIMAL && detail != VOPP_TREE_FULL))
    return fail(VOPP_E_INVALID, "bad tree detail");
  if (const int busy = check_not_pending(c)) return busy;
  c->tree_detail = detail;
  return VOPP_OK;
}

int vopp_ctx_set_option(vopp_ctx *c, int32_t option, int64_t value) {
  if (!c) return fail(VOPP_E_INVALID, "ctx is NULL");
  if (const int busy = check_not_pending(c)) return busy;
  switch (option) {
    case VOPP_OPT_LEAF_GEN: c->leaf_gen = value ? 1 : 0; return VOPP_OK;
    case VOPP_OPT_LEAF_THREADS:
      if (value < 32 || value > 256 || value % 32) return fail(VOPP_E_INVALID, "leaf threads");
      c->leaf_threads = (int)value;
      return VOPP_OK;
    case VOPP_OPT_GRID_CAP:
      if (value < 1) return fail(VOPP_E_INVALID, "grid cap");
      c->grid_cap = (int)std::min<int64_t>(value, 1 << 30);
      return VOPP_OK;
    case VOPP_OPT_PERSISTENT:
      if (value < 0 || value > 2) return fail(VOPP_E_INVALID, "persistent option %lld", (long long)value);
      c->leaf_persistent = (int)value;
      return VOPP_OK;
    case VOPP_OPT_FP64_ROOT: c->fp64_root = value ? 1 : 0; return VOPP_OK;
    case VOPP_OPT_GRAPHS:
      c->use_graphs = value ? 1 : 0;
      if (!c->use_graphs) c->graph.reset();
      return VOPP_OK;
    case VOPP_OPT_REUSE_COPY: c->reuse_copy = value ? 1 : 0; return VOPP_OK;
    case VOPP_OPT_SERVER_DIRECT: c->server_direct = value ? 1 : 0; return VOPP_OK;
    default: return fail(VOPP_E_INVALID, "unknown option %d", option);
  }
}

int vopp_ctx_set_timing(vopp_ctx *c, int enable) {
  if (!c) return fail(VOPP_E_INVALID, "ctx is NULL");
  if (const int busy = check_not_pending(c)) return busy;
  c->timing = enable != 0;
  return VOPP_OK;
}

int vopp_ctx_kernel_times(vopp_ctx *c, const char **names, double *ms, uint64_t *launches, int *n) {
  if (!c || !n) return fail(VOPP_E_INVALID, "NULL argument");
  const int m = std::min(*n, (int)F_ALL);
  for (int i = 0; i < m; ++i) {
    if (names) names[i] = kFamilies[i];
    if (ms) ms[i] = c->fam_ms[i];
    if (launches) launches[i] = c->fam_n[i];
  }
  *n = m;
  return VOPP_OK;
}

int vopp_ctx_reset_kernel_times(vopp_ctx *c) {
  if (!c) return fail(VOPP_E_INVALID, "ctx is NULL");
  for (int i = 0; i < F_ALL; ++i) { c->fam_ms[i] = 0; c->fam_n[i] = 0; }
  c->h2d_bytes = c->d2h_bytes = c->launches = 0;
  return VOPP_OK;
}

int vopp_ctx_counters(vopp_ctx *c, uint64_t *h2d_bytes, uint64_t *d2h_bytes, uint64_t *launches) {
  if (!c) return fail(VOPP_E_INVALID, "ctx is NULL");
  if (h2d_bytes) *h2d_bytes = c->h2d_bytes;
  if (d2h_bytes) *d2h_bytes = c->d2h_bytes;
  if (launches) *launches = c->launches;
  return VOPP_OK;
}

int vopp_plan_footprint(const vopp_model *m, int32_t N, int32_t D, int32_t W, size_t *bytes) {
  if (!m || !bytes) return fail(VOPP_E_INVALID, "NULL argument");
  int rc = validate_plan_args(m, N, D, W, 1.f, 0.5f, nullptr);
  if (rc) return rc;
  *bytes = make_layout(make_shape(m, N, D, W, m->ctx)).bytes;
  return VOPP_OK;
}

int vopp_create_model(vopp_ctx *c, const vopp_model_desc *d, vopp_model **out) {
  if (!c || !d || !out) return fail(VOPP_E_INVALID, "NULL argument");
  *out = nullptr;
  if (d->kind < VOPP_NAV2D || d->kind > VOPP_CROWD) return fail(VOPP_E_INVALID, "kind %d", d->kind);
  if (d->branch_mode != VOPP_BRANCH_SAMPLE && d->branch_mode != VOPP_BRANCH_ENUMERATE)
    return fail(VOPP_E_INVALID, "branch_mode");
  if (d->branch_mode == VOPP_BRANCH_ENUMERATE && d->kind == VOPP_NAV2D)
    return fail(VOPP_E_INVALID, "ENUMERATE needs a discrete observation space");
  if (d->pi_mode < VOPP_PI_UNIFORM || d->pi_mode > VOPP_PI_NAV_DIST)
    return fail(VOPP_E_INVALID, "pi_mode");
  if (d->pi_mode == VOPP_PI_NAV_DIST && (d->kind != VOPP_NAV2D || !(d->pi_temp > 0.f)))
    return fail(VOPP_E_INVALID, "NAV_DIST needs NAV2D and pi_temp > 0");
  const int A = d->kind == VOPP_NAV2D ? 4 : d->kind == VOPP_GRID ? 13 : d->kind == VOPP_CROWD ? 5 : 2;
  if (d->pi_mode == VOPP_PI_FIXED) {
    double s = 0.0;
    for (int a = 0; a < A; ++a) {
      if (!(d->pi_fixed[a] >= 0.f)) return fail(VOPP_E_INVALID, "pi_fixed[%d]", a);
      s += d->pi_fixed[a];
    }
    if (!(s > 0.0)) return fail(VOPP_E_INVALID, "pi_fixed sums to 0");
  }
  if (d->kind == VOPP_GRID) {
    for (int r = 0; r < 8; ++r) {
      const int x = d->rock_x[r], y = d->rock_y[r];
      if (x < 0 || x > 10 || y < 0 || y > 10) return fail(VOPP_E_INVALID, "rock %d off grid", r);
      if (x == 0 && y == 5) return fail(VOPP_E_INVALID, "rock %d on the start cell", r);
      for (int q = 0; q < r; ++q)
        if (d->rock_x[q] == x && d->rock_y[q] == y) return fail(VOPP_E_INVALID, "rocks %d,%d coincide", q, r);
    }
  }
  vopp_model *m = new (std::nothrow) vopp_model;
  if (!m) return fail(VOPP_E_NOMEM, "model alloc");
  m->ctx = c;
  m->desc = *d;
  m->A = A;
  DevModel &h = m->host;
  std::memset(&h, 0, sizeof h);
  h.kind = d->kind;
  h.A = A;
  h.n_obs = d->kind == VOPP_NAV2D ? 0 : (d->kind == VOPP_GRID ? 3 : (d->kind == VOPP_CROWD ? 64 : 2));
  h.branch_mode = d->branch_mode;
  h.pi_mode = d->pi_mode;
  h.h_zero = d->h_zero;
  h.pi_temp = d->pi_temp;
  if (d->kind == VOPP_GRID) fill_grid_tables(h, *d);
  h.toy_thr = (unsigned long long)std::floor(0.85 * 4294967296.0);
  h.toy_lc = (float)std::log(0.85);
  h.toy_lw = (float)std::log(0.15);
  h.toy_lc2 = (float)std::log2(0.85);
  h.toy_lw2 = (float)std::log2(0.15);
  h.toy_pc = 0.85f;
  h.toy_pw = 0.15f;
  cudaSetDevice(c->device);
  if (cudaMalloc(&m->dev, sizeof(DevModel)) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return fail(VOPP_E_NOMEM, "model device alloc");
  }
  if (cudaMemcpy(m->dev, &h, sizeof(DevModel), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(m->dev);
    delete m;
    return fail(VOPP_E_CUDA, "model upload");
  }
  *out = m;
  return VOPP_OK;
}

void vopp_model_destroy(vopp_model *m) {
  if (!m) return;
  cudaStreamSynchronize(m->ctx->stream);
  cudaFree(m->dev);
  delete m;
}

int vopp_model_num_actions(const vopp_model *m) {
  if (!m) return fail(VOPP_E_INVALID, "model is NULL");
  return m->A;
}

int vopp_grid_thresholds(uint64_t *thr, int32_t n) {
  if (!thr || n < 1 || n > kGridD2) return fail(VOPP_E_INVALID, "bad arguments");
  vopp_model_desc d;
  std::memset(&d, 0, sizeof d);
  for (int r = 0; r < 8; ++r) { d.rock_x[r] = r; d.rock_y[r] = 0; }
  DevModel *h = new (std::nothrow) DevModel;
  if (!h) return fail(VOPP_E_NOMEM, "host alloc");
  fill_grid_tables(*h, d);
  for (int i = 0; i < n; ++i) thr[i] = h->thr[i];
  delete h;
  return VOPP_OK;
}

int vopp_plan(vopp_model *m, const void *root_states, const float *root_weights, int32_t N,
              int32_t depth, int32_t width, float eta, float gamma, const float *pi_bar,
              uint64_t seed, uint32_t ptr_flags, vopp_plan_result *out) {
  vopp::NvtxRange nvtx_range("vopp_plan");
  if (!m || !out) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_ctx *c = m->ctx;
  vopp_plan_params p{depth, width, eta, gamma, seed, pi_bar};
  std::vector<Job> jobs(1);
  int rc = make_job(c, m, root_states, root_weights, N, p, ptr_flags, jobs[0]);
  if (rc) return rc;
  cudaSetDevice(c->device);
  return run_jobs(c, jobs, out, nullptr);
}

int vopp_plan_submit(vopp_model *m, const void *root_states, const float *root_weights,
                     int32_t N, int32_t depth, int32_t width, float eta, float gamma,
                     const float *pi_bar, uint64_t seed, uint32_t ptr_flags) {
  vopp::NvtxRange nvtx_range("vopp_plan_submit");
  if (!m) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_ctx *c = m->ctx;
  if (const int busy = check_not_pending(c)) return busy;
  vopp_plan_params p{depth, width, eta, gamma, seed, pi_bar};
  std::vector<Job> jobs(1);
  int rc = make_job(c, m, root_states, root_weights, N, p, ptr_flags, jobs[0]);
  if (rc) return rc;
  cudaSetDevice(c->device);
  rc = ensure_arena(c, place_jobs(jobs));
  if (rc) return rc;
  c->slot.stream = c->stream;
  rc = enqueue_jobs(c, c->slot, c->arena, jobs, c->timing, c->use_graphs ? &c->graph : nullptr);
  if (rc) return rc;
  c->pending_jobs = std::move(jobs);
  c->plan_pending = true;
  return VOPP_OK;
}

vopp_ctx *vopp_model_ctx(const vopp_model *m) { return m ? m->ctx : nullptr; }

int vopp_plan_finish(vopp_ctx *c, vopp_plan_result *out) {
  vopp::NvtxRange nvtx_range("vopp_plan_finish");
  if (!c || !out) return fail(VOPP_E_INVALID, "NULL argument");
  if (!c->plan_pending) return fail(VOPP_E_INVALID, "no submitted plan");
  c->plan_pending = false;
  cudaSetDevice(c->device);
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  timed_collect(c);
  const int rc = collect_results(c, c->slot, c->pending_jobs, out, nullptr, true);
  c->pending_jobs.clear();
  return rc;
}

int vopp_plan_anytime(vopp_model *m, const void *root_states, const float *root_weights,
                      int32_t N, const vopp_plan_params *p, double budget_s, uint32_t ptr_flags,
                      vopp_plan_result *out, int32_t *depth_reached) {
  vopp::NvtxRange nvtx_range("vopp_plan_anytime");
  if (!m || !p || !out) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_ctx *c = m->ctx;
  Job j;
  int rc = make_job(c, m, root_states, root_weights, N, *p, ptr_flags, j);
  if (rc) return rc;
  cudaSetDevice(c->device);
  return run_anytime(c, j, budget_s, out, depth_reached);
}

int vopp_plan_batch(vopp_ctx *c, int32_t n, const vopp_plan_request *reqs, vopp_plan_result *outs) {
  vopp::NvtxRange nvtx_range("vopp_plan_batch");
  if (!c || !reqs || !outs || n < 1) return fail(VOPP_E_INVALID, "bad batch arguments");
  std::vector<Job> jobs(n);
  for (int i = 0; i < n; ++i) {
    const vopp_plan_request &r = reqs[i];
    if (!r.model || r.model->ctx != c) return fail(VOPP_E_INVALID, "request %d: model of another context", i);
    int rc = make_job(c, r.model, r.root_states, r.root_weights, r.n_particles, r.params, r.ptr_flags, jobs[i]);
    if (rc) return rc;
  }
  cudaSetDevice(c->device);
  std::vector<int> st(n);
  int rc = run_jobs(c, jobs, outs, st.data());
  return rc;
}

int vopp_autotune(vopp_ctx *c, int32_t n, const vopp_plan_request *reqs, int32_t reps,
                  vopp_tune_result *out) {
  if (!c || !reqs || !out || n < 1 || reps < 1) return fail(VOPP_E_INVALID, "bad autotune arguments");
  if (const int busy = check_not_pending(c)) return busy;
  std::vector<Job> jobs(n);
  for (int i = 0; i < n; ++i) {
    const vopp_plan_request &r = reqs[i];
    if (!r.model || r.model->ctx != c) return fail(VOPP_E_INVALID, "request %d: model of another context", i);
    int rc = make_job(c, r.model, r.root_states, r.root_weights, r.n_particles, r.params, r.ptr_flags, jobs[i]);
    if (rc) return rc;
  }
  cudaSetDevice(c->device);
  const int threads[3] = {64, 128, 256};
  const int saved_threads = c->leaf_threads, saved_pers = c->leaf_persistent, saved_timing = c->timing;
  const bool saved_graphs = c->use_graphs;
  c->timing = false;
  c->use_graphs = 0;
  std::memset(out, 0, sizeof *out);
  std::vector<vopp_plan_result> ref(n), got(n);
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  double best = 1e300;
  int rc = VOPP_OK, k = 0;
  for (int pers = 0; pers < 2 && rc == VOPP_OK; ++pers) {
    for (int t = 0; t < 3 && rc == VOPP_OK; ++t, ++k) {
      c->leaf_threads = threads[t];
      c->leaf_persistent = pers;
      rc = run_jobs(c, jobs, k == 0 ? ref.data() : got.data(), nullptr);   // warm-up
      if (rc) break;
      if (k > 0) {   // configurations only reorder FP32 sums: results agree within 1e-4
        for (int i = 0; i < n; ++i) {
          const int A = jobs[i].shape.A;
          double top1 = -1e300, top2 = -1e300;
          for (int a = 0; a < A; ++a) {
            const double d = std::fabs(ref[i].q[a] - got[i].q[a]);
            if (d > 1e-4 * std::max(std::fabs(ref[i].q[a]), 1.0))
              rc = fail(VOPP_E_CUDA, "configuration changed a value beyond the tolerance");
            if (ref[i].q[a] > top1) { top2 = top1; top1 = ref[i].q[a]; }
            else if (ref[i].q[a] > top2) top2 = ref[i].q[a];
          }
          if (ref[i].action != got[i].action && top1 - top2 > 1e-4 * std::max(std::fabs(top1), 1.0))
            rc = fail(VOPP_E_CUDA, "configuration changed a clear action choice");
        }
        if (rc) break;
      }
      double ms_best = 1e300;
      for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, c->stream);
        rc = run_jobs(c, jobs, got.data(), nullptr);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_best = std::min(ms_best, (double)ms);
        if (rc) break;
      }
      out->tried_ms[k] = ms_best;
      out->tried_threads[k] = threads[t];
      out->tried_persistent[k] = pers;
      if (ms_best < best) {
        best = ms_best;
        out->leaf_threads = threads[t];
        out->persistent = pers;
      }
    }
  }
  out->n_tried = k;
  out->best_ms = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->timing = saved_timing;
  c->use_graphs = saved_graphs;
  if (rc != VOPP_OK) {
    c->leaf_threads = saved_threads;
    c->leaf_persistent = saved_pers;
    return rc;
  }
  c->leaf_threads = out->leaf_threads;   // keep the winner for the context
  c->leaf_persistent = out->persistent;
  c->graph.reset();
  return VOPP_OK;
}

int vopp_tree_read(vopp_ctx *c, int32_t field, int32_t level, uint64_t offset, uint64_t count,
                   void *dst, uint32_t ptr_flags) {
  return vopp_tree_read_plan(c, 0, field, level, offset, count, dst, ptr_flags);
}

int vopp_tree_read_plan(vopp_ctx *c, int32_t plan, int32_t field, int32_t level, uint64_t offset,
                        uint64_t count, void *dst, uint32_t ptr_flags) {
  if (!c || !dst) return fail(VOPP_E_INVALID, "NULL argument");
  if (const int busy = check_not_pending(c)) return busy;
  if (plan < 0 || plan >= (int)c->last_desc.size()) return fail(VOPP_E_INVALID, "no such plan");
  const PlanDesc &P = c->last_desc[plan];
  if (level < 0 || level > P.D) return fail(VOPP_E_INVALID, "level %d", level);
  const unsigned long long nodes = ipow(P.AW, level);
  const void *src = nullptr;
  size_t esz = 4;
  unsigned long long len = nodes;
  const int lv = level;
  switch (field) {
    case VOPP_FIELD_V: src = P.V[lv]; break;
    case VOPP_FIELD_Q: src = lv < kMaxDepth ? P.Q[lv] : nullptr; len = nodes * P.A; break;
    case VOPP_FIELD_RBAR: src = P.rbar[lv]; break;
    case VOPP_FIELD_LOMEGA: src = P.lom[lv]; break;
    case VOPP_FIELD_REP: src = P.rep[lv]; break;
    case VOPP_FIELD_OBS: src = P.obs[lv]; len = 2 * nodes; break;
    case VOPP_FIELD_PX: src = lv < kMaxDepth ? P.px[lv] : nullptr; len = nodes * P.N; break;
    case VOPP_FIELD_PY: src = lv < kMaxDepth ? P.py[lv] : nullptr; len = nodes * P.N; break;
    case VOPP_FIELD_PS: src = lv < kMaxDepth ? P.ps[lv] : nullptr; len = nodes * P.N; break;
    case VOPP_FIELD_PLW: src = lv < kMaxDepth ? P.plw[lv] : nullptr; len = nodes * P.N; break;
    case VOPP_FIELD_MU: src = lv < kMaxDepth ? P.mu[lv] : nullptr; len = 2 * nodes; break;
    case VOPP_FIELD_PSI: src = lv < kMaxDepth ? P.psi[lv] : nullptr; len = nodes * P.A; break;
    case VOPP_FIELD_PF: src = lv < kMaxDepth ? P.pf[lv] : nullptr; len = nodes * 12 * P.N; break;
    default: return fail(VOPP_E_INVALID, "field %d", field);
  }
  if (!src) return fail(VOPP_E_INVALID, "field %d not kept at level %d", field, level);
  if (offset > len || count > len - offset) return fail(VOPP_E_INVALID, "range outside the level");
  const cudaMemcpyKind kind = (ptr_flags & VOPP_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(cudaMemcpyAsync(dst, static_cast<const char *>(src) + offset * esz, count * esz, kind, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return VOPP_OK;
}

// ---- agents -----------------------------------------------------------------------------
int vopp_agent_create(vopp_model *m, const void *states, const float *weights, int32_t n,
                      uint64_t seed, uint32_t ptr_flags, vopp_agent **out) {
  if (!m || !states || !out) return fail(VOPP_E_INVALID, "NULL argument");
  if (n < 1 || n > VOPP_MAX_PARTICLES) return fail(VOPP_E_INVALID, "n %d", n);
  *out = nullptr;
  vopp_ctx *c = m->ctx;
  cudaSetDevice(c->device);
  const bool nav = m->desc.kind == VOPP_NAV2D;
  const bool dev = ptr_flags & VOPP_PTR_DEVICE;
  std::vector<float> lw(n);
  std::vector<float> wtmp;
  const float *w = weights;
  if (weights && dev) {
    wtmp.resize(n);
    CUDA_TRY(cudaMemcpy(wtmp.data(), weights, 4 * (size_t)n, cudaMemcpyDeviceToHost));
    w = wtmp.data();
  }
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const double wi = w ? w[i] : 1.0;
    if (!(wi >= 0.0)) return fail(VOPP_E_INVALID, "weight %d", i);
    s += wi;
  }
  if (!(s > 0.0)) return fail(VOPP_E_DEGENERATE, "weights sum to 0");
  if (m->desc.kind == VOPP_GRID) {
    std::vector<int32_t> stmp;
    const void *sh = states;
    if (dev) {
      stmp.resize(n);
      CUDA_TRY(cudaMemcpy(stmp.data(), states, 4 * (size_t)n, cudaMemcpyDeviceToHost));
      sh = stmp.data();
    }
    const int rc = check_grid_states(m, sh, n);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    const double wi = w ? w[i] : 1.0;
    lw[i] = wi > 0.0 ? (float)std::log(wi / s) : -INFINITY;
  }
  vopp_agent *g = new (std::nothrow) vopp_agent;
  if (!g) return fail(VOPP_E_NOMEM, "agent alloc");
  g->model = m;
  g->N = n;
  g->seed = seed;
  bool ok = true;
  // agent memory comes from the stream-ordered pool: creating or destroying an agent never
  // synchronises the device (a serving loop keeps running while agents come and go)
  cudaStream_t cs = c->stream;
  auto al = [&](void **p, size_t b) {
    if (ok && cudaMallocFromPoolAsync(p, b, c->pool, cs) != cudaSuccess) { cudaGetLastError(); ok = false; }
  };
  const int kind = m->desc.kind;
  const size_t words = root_words(kind);
  float *blk = nullptr, *tblk = nullptr;      // root_words(kind) rows of n words
  al((void **)&blk, 4 * words * (size_t)n);
  al((void **)&tblk, 4 * words * (size_t)n);
  if (ok) {
    if (nav || kind == kCrowd) { g->xy = blk; g->txy = tblk; }
    if (kind == kCrowd) {
      g->pf = blk + 2 * (size_t)n; g->tpf = tblk + 2 * (size_t)n;
      g->s = reinterpret_cast<int *>(blk + 14 * (size_t)n);
      g->ts = reinterpret_cast<int *>(tblk + 14 * (size_t)n);
    } else if (!nav) {
      g->s = reinterpret_cast<int *>(blk);
      g->ts = reinterpret_cast<int *>(tblk);
    }
    g->blk = blk;
    g->tblk = tblk;
  } else {
    if (blk) cudaFreeAsync(blk, cs);
    if (tblk) cudaFreeAsync(tblk, cs);
  }
  al((void **)&g->lw, 4 * (size_t)n);
  al((void **)&g->tlw, 4 * (size_t)n);
  al((void **)&g->cdf, 8 * (size_t)n);
  al((void **)&g->anc, 4 * (size_t)n);
  al((void **)&g->dout, sizeof(BeliefOut));
  if (!ok) { vopp_agent_destroy(g); return fail(VOPP_E_NOMEM, "agent device alloc"); }
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(g->blk, states, 4 * words * (size_t)n, k, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g->lw, lw.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);   // lw is a local buffer
  if (e != cudaSuccess) { vopp_agent_destroy(g); return fail(VOPP_E_CUDA, "agent upload: %s", cudaGetErrorString(e)); }
  *out = g;
  return VOPP_OK;
}

// ---- environment and closed loop ------------------------------------------------------
int vopp_env_create(vopp_model *m, const void *state, uint64_t seed, vopp_env **out) {
  if (!m || !state || !out) return fail(VOPP_E_INVALID, "NULL argument");
  *out = nullptr;
  if (const int rc = check_grid_states(m, state, 1)) return rc;
  vopp_ctx *c = m->ctx;
  cudaSetDevice(c->device);
  vopp_env *e = new (std::nothrow) vopp_env;
  if (!e) return fail(VOPP_E_NOMEM, "env alloc");
  e->model = m;
  e->seed = seed;
  const int kind = m->desc.kind;
  const size_t words = root_words(kind);     // the state as one particle of the root layout
  cudaError_t ce = cudaMalloc(&e->blk, 4 * words);
  if (ce == cudaSuccess) {
    if (kind == kNav || kind == kCrowd) e->xy = e->blk;
    if (kind == kCrowd) { e->pf = e->blk + 2; e->s = reinterpret_cast<int *>(e->blk + 14); }
    else if (kind != kNav) e->s = reinterpret_cast<int *>(e->blk);
  }
  if (ce == cudaSuccess) ce = cudaMalloc(&e->dout, sizeof(EnvOut));
  if (ce == cudaSuccess) ce = cudaMallocHost(&e->hout, sizeof(EnvOut));
  if (ce == cudaSuccess) ce = cudaMemcpy(e->blk, state, 4 * words, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    vopp_env_destroy(e);
    return fail(VOPP_E_NOMEM, "env buffers: %s", cudaGetErrorString(ce));
  }
  *out = e;
  return VOPP_OK;
}

int vopp_env_step(vopp_env *e, int32_t action, void *obs, float *reward, int32_t *terminal) {
  if (!e || !obs) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_model *m = e->model;
  if (action < 0 || action >= m->A) return fail(VOPP_E_INVALID, "action %d", action);
  vopp_ctx *c = m->ctx;
  cudaSetDevice(c->device);
  EnvArgs E;
  std::memset(&E, 0, sizeof E);
  E.kind = m->desc.kind;
  E.action = action;
  E.key0 = (uint32_t)e->seed;
  E.key1 = (uint32_t)(e->seed >> 32);
  E.t = e->t;
  E.xy = e->xy;
  E.s = e->s;
  E.pf = e->pf;
  E.model = m->dev;
  E.out = e->dout;
  cudaError_t ce = launch_env(E, c->stream);
  c->launches += 1;
  if (ce != cudaSuccess) return fail(VOPP_E_CUDA, "env launch: %s", cudaGetErrorString(ce));
  CUDA_TRY(cudaMemcpyAsync(e->hout, e->dout, sizeof(EnvOut), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (E.kind == kNav) {
    static_cast<float *>(obs)[0] = e->hout->obs[0];
    static_cast<float *>(obs)[1] = e->hout->obs[1];
  } else {
    *static_cast<int32_t *>(obs) = e->hout->obs_i;
  }
  if (reward) *reward = e->hout->reward;
  if (terminal) *terminal = e->hout->terminal;
  e->t += 1;
  return VOPP_OK;
}

int vopp_env_get_state(vopp_env *e, void *state) {
  if (!e || !state) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_ctx *c = e->model->ctx;
  cudaSetDevice(c->device);
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(cudaMemcpy(state, e->blk, 4 * root_words(e->model->desc.kind), cudaMemcpyDeviceToHost));
  return VOPP_OK;
}

void vopp_env_destroy(vopp_env *e) {
  if (!e) return;
  if (e->model) cudaStreamSynchronize(e->model->ctx->stream);
  cudaFree(e->blk); cudaFree(e->dout);
  if (e->hout) cudaFreeHost(e->hout);
  delete e;
}

int vopp_run_episode(vopp_agent *g, vopp_env *e, const vopp_plan_params *p, int32_t max_steps,
                     int32_t anytime, double budget_s, vopp_episode_result *out,
                     int32_t *actions, float *rewards) {
  if (!g || !e || !p || !out) return fail(VOPP_E_INVALID, "NULL argument");
  if (g->model != e->model) return fail(VOPP_E_INVALID, "agent and environment use different models");
  if (max_steps < 0) return fail(VOPP_E_INVALID, "max_steps %d", max_steps);
  std::memset(out, 0, sizeof *out);
  double disc = 1.0;
  for (int t = 0; t < max_steps; ++t) {
    vopp_plan_params pt = *p;
    pt.seed = p->seed + (uint64_t)t;
    vopp_plan_result r;
    const auto t0 = std::chrono::steady_clock::now();
    int32_t depth = pt.depth;
    int rc = anytime ? vopp_agent_plan_anytime(g, &pt, budget_s, &r, &depth)
                     : vopp_agent_plan(g, &pt, &r);
    out->plan_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rc) { out->status = rc; return rc; }
    out->particle_steps += r.particle_steps;
    if (t == 0 || depth < out->min_depth) out->min_depth = depth;
    float obs[2] = {0.f, 0.f};
    float rew = 0.f;
    int32_t term = 0;
    rc = vopp_env_step(e, r.action, obs, &rew, &term);
    if (rc) { out->status = rc; return rc; }
    if (actions) actions[t] = r.action;
    if (rewards) rewards[t] = rew;
    out->steps = t + 1;
    out->total_reward += rew;
    out->discounted_return += disc * rew;
    disc *= (double)p->gamma;
    if (term) { out->terminated = 1; break; }
    rc = vopp_belief_update(g, r.action, obs, nullptr, nullptr);
    if (rc) { out->status = rc; return rc; }
  }
  return VOPP_OK;
}

void vopp_agent_destroy(vopp_agent *g) {
  if (!g) return;
  if (g->model) {   // stream-ordered frees: no device-wide synchronisation
    cudaStream_t s = g->model->ctx->stream;
    free_kept(g->tree, s);
    free_kept(g->sub, s);
    for (void *p : {(void *)g->blk, (void *)g->tblk, (void *)g->lw, (void *)g->tlw,
                    (void *)g->cdf, (void *)g->anc, (void *)g->dout, (void *)g->spare})
      if (p) cudaFreeAsync(p, s);
    if (g->spare_ev) cudaEventDestroy(g->spare_ev);
  }
  delete g;
}

int vopp_agent_num_particles(const vopp_agent *g) {
  if (!g) return fail(VOPP_E_INVALID, "agent is NULL");
  return g->N;
}

int vopp_agent_plan(vopp_agent *g, const vopp_plan_params *p, vopp_plan_result *out) {
  vopp::NvtxRange nvtx_range("vopp_agent_plan");
  if (!g || !p || !out) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_ctx *c = g->model->ctx;
  std::vector<Job> jobs(1);
  const void *states = g->blk;
  int rc = make_job(c, g->model, states, nullptr, g->N, *p, VOPP_PTR_DEVICE, jobs[0]);
  if (rc) return rc;
  jobs[0].log_weights = g->lw;
  cudaSetDevice(c->device);
  if (!g->reuse) return run_jobs(c, jobs, out, nullptr);
  Job &j = jobs[0];
  attach_reuse(g, j);
  j.own_arena = take_spare(g, j.lay.bytes);
  if (!j.own_arena &&
      cudaMallocFromPoolAsync(reinterpret_cast<void **>(&j.own_arena), j.lay.bytes, c->pool, c->stream) !=
          cudaSuccess) {
    cudaGetLastError();
    return fail(VOPP_E_NOMEM, "plan memory for the kept tree");
  }
  rc = run_jobs(c, jobs, out, nullptr);
  keep_tree(g, j, rc == VOPP_OK, c->stream);
  return rc;
}

int vopp_agent_set_reuse(vopp_agent *g, int32_t enable) {
  if (!g) return fail(VOPP_E_INVALID, "agent is NULL");
  if (enable < 0 || enable > 2) return fail(VOPP_E_INVALID, "enable must be 0, 1 or 2");
  // continuous observations (NAV2D) practically never equal a branch's sampled one: a kept
  // tree would cost every plan its memory and observation stores for nothing
  g->reuse = enable == 2 || (enable == 1 && g->model->desc.kind != VOPP_NAV2D);
  if (!g->reuse) {
    cudaStream_t s = g->model->ctx->stream;
    free_kept(g->tree, s);
    free_kept(g->sub, s);
    if (g->spare) cudaFreeAsync(g->spare, s);
    g->spare = nullptr;
    g->spare_bytes = 0;
    g->adopted_slot = -1;
  }
  return VOPP_OK;
}

int vopp_agent_reuse_info(const vopp_agent *g, int32_t *adopted_slot, int32_t *kept_levels,
                          int32_t *key_level) {
  if (!g) return fail(VOPP_E_INVALID, "agent is NULL");
  if (adopted_slot) *adopted_slot = g->sub ? g->adopted_slot : -1;
  if (kept_levels) *kept_levels = g->sub ? g->sub->shape.mat_top + 1 : 0;
  if (key_level) *key_level = g->sub ? g->sub->lvl_off : 0;
  return VOPP_OK;
}

int vopp_agent_plan_anytime(vopp_agent *g, const vopp_plan_params *p, double budget_s,
                            vopp_plan_result *out, int32_t *depth_reached) {
  if (!g || !p || !out) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_ctx *c = g->model->ctx;
  Job j;
  const void *states = g->blk;
  int rc = make_job(c, g->model, states, nullptr, g->N, *p, VOPP_PTR_DEVICE, j);
  if (rc) return rc;
  j.log_weights = g->lw;
  cudaSetDevice(c->device);
  return run_anytime(c, j, budget_s, out, depth_reached);
}

int vopp_agent_plan_episodes(vopp_agent *g, const vopp_episode_params *p, double budget_s,
                             vopp_plan_result *out, int32_t *depth_reached, int32_t *n_nodes) {
  if (!g || !p || !out) return fail(VOPP_E_INVALID, "NULL argument");
  const void *states = g->blk;
  vopp::EpisodeInputs in{states, nullptr, g->lw, g->N, VOPP_PTR_DEVICE};
  return vopp::run_plan_episodes(g->model, in, *p, budget_s, out, depth_reached, n_nodes);
}

}  // extern "C"

namespace {

// The SIR kernel's arguments for agent g under (action, obs); obs is a host pointer (NAV2D
// float[2], other models int32[1]).  The result goes to `out` (device).
BeliefArgs belief_args(vopp_agent *g, int32_t action, const void *obs, BeliefOut *out) {
  const vopp_model *m = g->model;
  BeliefArgs B;
  std::memset(&B, 0, sizeof B);
  B.kind = m->desc.kind;
  B.N = g->N;
  B.action = action;
  B.key0 = (uint32_t)g->seed;
  B.key1 = (uint32_t)(g->seed >> 32);
  B.t = g->t;
  if (B.kind == kNav || B.kind == kCrowd) {
    B.x = g->xy; B.y = g->xy + g->N; B.tx = g->txy; B.ty = g->txy + g->N;
  }
  if (B.kind == kNav) {
    const float *o = static_cast<const float *>(obs);
    B.obs_f[0] = o[0];
    B.obs_f[1] = o[1];
  } else {
    B.s = g->s; B.ts = g->ts;
    B.pf = g->pf; B.tpf = g->tpf;
    B.obs_i = *static_cast<const int32_t *>(obs);
  }
  B.lw = g->lw;
  B.tlw = g->tlw;
  B.cdf = g->cdf;
  B.anc = g->anc;
  B.model = m->dev;
  B.out = out;
  return B;
}

// Subtree reuse at a belief update: adopt the matching branch of the kept tree (slot >= 0,
// its subtree kept) or release what the agent kept (slot < 0: the SIR update follows).
int reuse_update(vopp_agent *g, int slot, cudaStream_t s) {
  release_kept(g, g->sub, s);
  g->adopted_slot = -1;
  if (slot < 0) {
    release_kept(g, g->tree, s);
    return VOPP_OK;
  }
  const int rc = adopt_subtree(g, slot, s);
  release_kept(g, g->tree, s);
  if (rc) return rc;
  g->adopted_slot = slot;
  return VOPP_OK;
}

}  // namespace

extern "C" {

int vopp_belief_update(vopp_agent *g, int32_t action, const void *obs, double *ess_out,
                       int32_t *resampled_out) {
  vopp::NvtxRange nvtx_range("vopp_belief_update");
  if (!g || !obs) return fail(VOPP_E_INVALID, "NULL argument");
  vopp_model *m = g->model;
  if (action < 0 || action >= m->A) return fail(VOPP_E_INVALID, "action %d", action);
  vopp_ctx *c = m->ctx;
  cudaSetDevice(c->device);
  BeliefArgs B = belief_args(g, action, obs, g->dout);
  if (g->reuse) {
    // subtree reuse: a kept tree's branch of this action that sampled this very observation
    // becomes the belief (its particle set, as the tree holds it), and its subtree is kept
    const int slot = matching_branch(g, action, B.obs_f, B.obs_i, c->stream);
    const int rc = reuse_update(g, slot, c->stream);
    if (rc) return rc;
    if (slot >= 0) {
      CUDA_TRY(cudaStreamSynchronize(c->stream));
      g->t += 1;
      if (ess_out) *ess_out = -1.0;
      if (resampled_out) *resampled_out = 0;
      return VOPP_OK;
    }
  }
  TimedLaunch tl;
  timed_begin(c, F_BELIEF, tl);
  cudaError_t e = launch_belief(B, c->stream);
  c->launches += 1;
  c->d2h_bytes += sizeof(BeliefOut);
  timed_end(c, tl);
  if (e != cudaSuccess) return fail(VOPP_E_CUDA, "belief launch: %s", cudaGetErrorString(e));
  CUDA_TRY(cudaMemcpyAsync(&g->hout, g->dout, sizeof(BeliefOut), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  timed_collect(c);
  if (g->hout.status) return fail(VOPP_E_DEGENERATE, "observation has zero likelihood under every particle");
  if (ess_out) *ess_out = g->hout.ess;
  if (resampled_out) *resampled_out = g->hout.resampled;
  g->t += 1;
  return VOPP_OK;
}

int vopp_belief_update_batch(vopp_ctx *c, int32_t n, vopp_agent *const *agents,
                             const int32_t *actions, const void *const *obs, double *ess_out,
                             int32_t *resampled_out, int32_t *status_out) {
  vopp::NvtxRange nvtx_range("vopp_belief_update_batch");
  if (!c || n < 0) return fail(VOPP_E_INVALID, "bad batch arguments");
  if (n == 0) return VOPP_OK;
  if (!agents || !actions || !obs || !status_out) return fail(VOPP_E_INVALID, "NULL argument");
  {
    std::vector<const vopp_agent *> seen(agents, agents + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(VOPP_E_INVALID, "an agent appears twice in the batch");
  }
  for (int i = 0; i < n; ++i) {
    const vopp_agent *g = agents[i];
    if (!g || !obs[i]) return fail(VOPP_E_INVALID, "NULL agent or observation at %d", i);
    if (g->model->ctx != c) return fail(VOPP_E_INVALID, "agent %d belongs to another context", i);
    if (actions[i] < 0 || actions[i] >= g->model->A) return fail(VOPP_E_INVALID, "action %d at %d", actions[i], i);
  }
  cudaSetDevice(c->device);
  cudaStream_t s = c->stream;
  std::vector<BeliefArgs> args(n);
  for (int i = 0; i < n; ++i) args[i] = belief_args(agents[i], actions[i], obs[i], nullptr);

  // subtree reuse: the kept trees' level-1 observations and branch weights of the agents'
  // actions, one copy each and one synchronisation for all, then adoptions (a branch whose
  // particles all have zero weight, log omega = -inf, is never adopted)
  std::vector<int> slot(n, -1);
  {
    std::vector<int> asked;
    std::vector<float> ob, lo;
    std::vector<size_t> at(n, 0), atl(n, 0);
    for (int i = 0; i < n; ++i) {
      const KeptTree *t = agents[i]->reuse ? agents[i]->tree : nullptr;
      if (!t || t->shape.mat_top < 1 || t->lay.obs[1] == kNone) continue;
      at[i] = ob.size();
      ob.resize(ob.size() + 2 * (size_t)t->shape.W);
      atl[i] = lo.size();
      lo.resize(lo.size() + (size_t)t->shape.W, 0.0f);
      asked.push_back(i);
    }
    for (int i : asked) {
      const KeptTree *t = agents[i]->tree;
      CUDA_TRY(cudaMemcpyAsync(ob.data() + at[i], t->mem + t->lay.obs[1] + 8 * (size_t)actions[i] * t->shape.W,
                               8 * (size_t)t->shape.W, cudaMemcpyDeviceToHost, s));
      if (t->lay.lom[1] != kNone)
        CUDA_TRY(cudaMemcpyAsync(lo.data() + atl[i], t->mem + t->lay.lom[1] + 4 * (size_t)actions[i] * t->shape.W,
                                 4 * (size_t)t->shape.W, cudaMemcpyDeviceToHost, s));
    }
    if (!asked.empty()) CUDA_TRY(cudaStreamSynchronize(s));
    for (int i : asked) {
      const KeptTree *t = agents[i]->tree;
      for (int k = 0; k < t->shape.W; ++k) {
        const float *o = ob.data() + at[i] + 2 * k;
        const bool eq = (t->shape.kind == kNav) ? (o[0] == args[i].obs_f[0] && o[1] == args[i].obs_f[1])
                                                : ((int)o[0] == args[i].obs_i);
        if (eq) {
          if (lo[atl[i] + k] > -INFINITY) slot[i] = actions[i] * t->shape.W + k;
          break;
        }
      }
    }
    for (int i = 0; i < n; ++i) {
      status_out[i] = VOPP_OK;
      if (!agents[i]->reuse) continue;
      const int rc = reuse_update(agents[i], slot[i], s);
      if (rc) { status_out[i] = rc; slot[i] = -2; }   // failed adoption: no update
    }
  }

  // SIR for every other agent: one CTA each in one launch
  std::vector<int> sir;
  for (int i = 0; i < n; ++i) if (slot[i] == -1) sir.push_back(i);
  const int ns = (int)sir.size();
  std::vector<BeliefOut> hres(ns);
  if (ns > 0) {
    char *mem = nullptr;
    const size_t res_off = align_up(sizeof(BeliefArgs) * ns, 256);
    if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(&mem), res_off + sizeof(BeliefOut) * ns, c->pool, s) !=
        cudaSuccess) {
      cudaGetLastError();
      return fail(VOPP_E_NOMEM, "batch arguments");
    }
    BeliefArgs *dargs = reinterpret_cast<BeliefArgs *>(mem);
    BeliefOut *dres = reinterpret_cast<BeliefOut *>(mem + res_off);
    std::vector<BeliefArgs> sargs(ns);
    for (int q = 0; q < ns; ++q) { sargs[q] = args[sir[q]]; sargs[q].out = dres + q; }
    TimedLaunch tl;
    timed_begin(c, F_BELIEF, tl);
    cudaError_t e = cudaMemcpyAsync(dargs, sargs.data(), sizeof(BeliefArgs) * ns, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_belief_batch(dargs, ns, s);
    timed_end(c, tl);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hres.data(), dres, sizeof(BeliefOut) * ns, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(mem, s);
    c->launches += 1;
    c->h2d_bytes += sizeof(BeliefArgs) * ns;
    c->d2h_bytes += sizeof(BeliefOut) * ns;
    if (e != cudaSuccess) return fail(VOPP_E_CUDA, "batched belief update: %s", cudaGetErrorString(e));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  timed_collect(c);
  for (int i = 0; i < n; ++i) {
    if (ess_out) ess_out[i] = 0.0;
    if (resampled_out) resampled_out[i] = 0;
    if (slot[i] >= 0) {                    // adopted
      agents[i]->t += 1;
      if (ess_out) ess_out[i] = -1.0;
    }
  }
  int first = VOPP_OK;
  for (int q = 0; q < ns; ++q) {
    const int i = sir[q];
    if (hres[q].status) {
      status_out[i] = VOPP_E_DEGENERATE;
    } else {
      agents[i]->t += 1;
      if (ess_out) ess_out[i] = hres[q].ess;
      if (resampled_out) resampled_out[i] = hres[q].resampled;
    }
  }
  for (int i = 0; i < n; ++i) if (status_out[i] && !first) first = status_out[i];
  if (first) return fail(first, "belief update failed for some agents (see status_out)");
  return VOPP_OK;
}

int vopp_agent_get_particles(vopp_agent *g, void *states, float *log_weights, int32_t *ancestors,
                             uint32_t ptr_flags) {
  if (!g) return fail(VOPP_E_INVALID, "agent is NULL");
  vopp_ctx *c = g->model->ctx;
  const cudaMemcpyKind k = (ptr_flags & VOPP_PTR_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t n = (size_t)g->N;
  if (states)
    CUDA_TRY(cudaMemcpyAsync(states, g->blk, 4 * root_words(g->model->desc.kind) * n, k, c->stream));
  if (log_weights) CUDA_TRY(cudaMemcpyAsync(log_weights, g->lw, 4 * n, k, c->stream));
  if (ancestors) CUDA_TRY(cudaMemcpyAsync(ancestors, g->anc, 4 * n, k, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return VOPP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Serving loop: continuous batching of plan requests.
//
// Requests wait in a FIFO.  A worker thread forms a batch from the head of the queue
// whenever a slot is free and the HBM budget admits it, builds the batch's launch sequence
// on the slot's own stream (arena from the device's stream-ordered pool, released on the
// same stream after the results are copied back) and records an event after it.  While any
// batch is in flight the worker polls the slots' events and the queue (yielding the CPU
// between polls), so a finished batch is posted and a new request is started within
// microseconds; with nothing in flight it sleeps on a condition variable.  The server mutex
// guards only the queue, the results and the counters: the worker releases it around its
// CUDA calls, so callers that submit or collect are never held up by a launch.  Batches on
// different slots run concurrently on the device, and requests that arrive while others run
// join the next batch.  Each plan's random numbers are keyed by its own seed, so a plan's
// result does not depend on which batch it joined.
// ---------------------------------------------------------------------------------------
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// A short pause for spin loops (no system call).
inline void cpu_relax() {
#if defined(__x86_64__) || defined(__i386__)
  __builtin_ia32_pause();
#elif defined(__aarch64__)
  asm volatile("yield");
#endif
}

// Waits of at most this long spin instead of sleeping on the condition variable (a serving
// loop that waits for its next completion or arrival sees either within a microsecond; a
// sleeping thread would pay a wake-up, tens of microseconds, on every request).
constexpr double kSpinWaitMax = 5e-3;

struct ServerReq {
  uint64_t ticket = 0;
  Job job;
  std::vector<char> host_states, host_weights;   // copies of host inputs
  std::vector<float> pi_bar;
  size_t bytes = 0;
  double t_submit = 0.0;
};

// A slot is claimed (busy set) under the server mutex by the thread that launches its batch:
// the worker, or a submitting thread that found the server idle.  While `launching` is set
// only that thread touches the slot; afterwards only the worker does, until it posts the
// batch and clears busy.
struct ServerSlot {
  Slot slot;
  GraphSet graphs;                 // the slot's replayable launch sequences (server graphs on)
  cudaEvent_t done_ev = nullptr;   // recorded after the batch's last operation
  char *arena = nullptr;
  size_t arena_bytes = 0;
  // the slot's plan memory, kept between batches (the slot's stream orders its batches) so
  // that a batch that fits needs no allocation; larger batches replace it up to kSlotKeepMax
  char *kept = nullptr;
  size_t kept_bytes = 0;
  std::vector<ServerReq> reqs;
  std::vector<Job> jobs;
  std::atomic<bool> busy{false};
  std::atomic<bool> launching{false};   // claimed, batch not yet enqueued (worker: hands off)
};

struct Done {
  int status;
  vopp_plan_result res;
  double t_submit, t_done;
};

}  // namespace

struct vopp_server {
  vopp_ctx *c = nullptr;
  int max_batch = 64;
  int use_graphs = 0;              // replay recorded launch sequences (VOPP_OPT_GRAPHS at creation)
  bool direct = false;             // an idle server's submitting thread launches the request
  size_t budget = 0, in_flight = 0, peak_in_flight = 0;
  std::vector<ServerSlot *> slots;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::atomic<bool> stop_flag{false};   // stop, readable without the lock
  bool paused = false;          // queue requests without starting batches
  std::deque<ServerReq> pending;
  std::atomic<size_t> n_pending{0};   // pending.size(), readable without the lock
  std::unordered_map<uint64_t, Done> done;
  std::deque<uint64_t> completion_order;   // tickets in the order their plans finished
  std::atomic<size_t> n_order{0};          // completion_order.size(), readable without the lock
  uint64_t next_ticket = 1;
  vopp_server_stats stats{};
  int worker_error = VOPP_OK;
};

namespace {

// Batches of at most this many particle-steps (about a fifth of a millisecond of leaf work
// for the navigation model) count as small for the choice of stream priority.
constexpr double kSmallBatchSteps = 3.0e7;

vopp_plan_result failed_result() {
  vopp_plan_result z;
  std::memset(&z, 0, sizeof z);
  z.action = -1;
  return z;
}

// Post a status for every request of a batch (lock held).
void post_failure(vopp_server *srv, std::vector<ServerReq> &batch, int rc) {
  const double t = now_s();
  for (auto &r : batch) {
    srv->done[r.ticket] = Done{rc, failed_result(), r.t_submit, t};
    srv->completion_order.push_back(r.ticket);
  }
  srv->n_order.store(srv->completion_order.size());
}

// A finished slot's outcomes, gathered without the lock (worker thread): the results are
// in the slot's pinned mirror (the stream copied them back before the slot's event), and
// agents that keep their trees take their plan's memory.
struct Harvest {
  std::vector<std::pair<uint64_t, Done>> done;
  unsigned long long steps = 0;
  int completed = 0;
};
Harvest gather(vopp_server *srv, ServerSlot *s, bool ok) {
  Harvest h;
  const int n = (int)s->jobs.size();
  const double t = now_s();
  if (ok) {
    std::vector<vopp_plan_result> outs(n);
    std::vector<int> st(n);
    collect_results(srv->c, s->slot, s->jobs, outs.data(), st.data(), false);
    for (int i = 0; i < n; ++i) {
      if (s->jobs[i].agent) keep_tree(s->jobs[i].agent, s->jobs[i], st[i] == VOPP_OK, s->slot.stream);
      h.done.emplace_back(s->reqs[i].ticket, Done{st[i], outs[i], s->reqs[i].t_submit, t});
      h.steps += outs[i].particle_steps;
    }
    h.completed = n;
  } else {
    for (auto &j : s->jobs)
      if (j.agent) keep_tree(j.agent, j, false, s->slot.stream);
    for (auto &r : s->reqs) h.done.emplace_back(r.ticket, Done{VOPP_E_CUDA, failed_result(), r.t_submit, t});
  }
  return h;
}

// Post a gathered slot and free the slot (lock held).
void post(vopp_server *srv, ServerSlot *s, Harvest &h) {
  for (auto &d : h.done) {
    srv->done[d.first] = d.second;
    srv->completion_order.push_back(d.first);
  }
  srv->n_order.store(srv->completion_order.size());
  srv->stats.completed += h.completed;
  srv->stats.particle_steps += h.steps;
  srv->in_flight -= s->arena_bytes;
  s->arena = nullptr;
  s->arena_bytes = 0;
  s->reqs.clear();
  s->jobs.clear();
  s->busy = false;
}

// Take a batch from the head of the queue within the budget and reserve its bytes (lock
// held).  A request that could never fit is refused at once.
std::vector<ServerReq> take_batch(vopp_server *srv, size_t *bytes_out) {
  std::vector<ServerReq> batch;
  size_t bytes = 0;
  while (!srv->pending.empty() && (int)batch.size() < srv->max_batch) {
    ServerReq &r = srv->pending.front();
    if (srv->in_flight + bytes + r.bytes > srv->budget) {
      if (batch.empty() && srv->in_flight == 0) {   // can never fit: refuse it
        srv->done[r.ticket] = Done{VOPP_E_BUDGET, failed_result(), r.t_submit, now_s()};
        srv->completion_order.push_back(r.ticket);
        srv->n_order.store(srv->completion_order.size());
        srv->stats.rejected += 1;
        srv->pending.pop_front();
        continue;
      }
      break;
    }
    bytes += r.bytes;
    batch.push_back(std::move(r));
    srv->pending.pop_front();
  }
  srv->in_flight += bytes;
  srv->n_pending.store(srv->pending.size());
  *bytes_out = bytes;
  return batch;
}

// The most plan memory a slot keeps between batches.
constexpr size_t kSlotKeepMax = size_t(256) << 20;

// Enqueue a batch on a slot's stream (worker thread, lock NOT held).
int launch_batch(vopp_server *srv, ServerSlot *s, std::vector<ServerReq> &batch) {
  std::vector<Job> jobs;
  for (auto &r : batch) {
    jobs.push_back(r.job);
    Job &j = jobs.back();
    if (!r.host_states.empty()) j.states = r.host_states.data();
    if (!r.host_weights.empty()) j.weights = reinterpret_cast<const float *>(r.host_weights.data());
    if (!r.pi_bar.empty()) j.p.pi_bar = r.pi_bar.data();
  }
  const size_t arena_bytes = place_jobs(jobs);
  char *arena = nullptr;
  cudaError_t e = cudaSuccess;
  bool own = false;                         // a one-off arena, released after the batch
  if (arena_bytes <= s->kept_bytes) {
    arena = s->kept;
  } else {
    if (s->kept) cudaFreeAsync(s->kept, s->slot.stream);
    s->kept = nullptr;
    s->kept_bytes = 0;
    e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&arena), arena_bytes, srv->c->pool,
                                s->slot.stream);
    if (e == cudaSuccess && arena_bytes <= kSlotKeepMax) {
      s->kept = arena;
      s->kept_bytes = arena_bytes;
    } else {
      own = e == cudaSuccess;
    }
  }
  for (auto &j : jobs)   // plans whose agents keep their trees get memory of their own
    if (e == cudaSuccess && j.agent && !(j.own_arena = take_spare(j.agent, j.lay.bytes)))
      e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&j.own_arena), j.lay.bytes, srv->c->pool,
                                  s->slot.stream);
  int rc = (e == cudaSuccess) ? enqueue_jobs(srv->c, s->slot, arena, jobs, false,
                                             srv->use_graphs ? &s->graphs : nullptr)
                               : VOPP_E_NOMEM;
  if (rc == VOPP_OK) {
    if ((own && cudaFreeAsync(arena, s->slot.stream) != cudaSuccess) ||
        cudaEventRecord(s->done_ev, s->slot.stream) != cudaSuccess)
      rc = VOPP_E_CUDA;
  }
  if (rc != VOPP_OK) {
    cudaGetLastError();
    if (own) cudaFreeAsync(arena, s->slot.stream);
    for (auto &j : jobs)
      if (j.own_arena) cudaFreeAsync(j.own_arena, s->slot.stream);
    cudaStreamSynchronize(s->slot.stream);
    return rc;
  }
  s->arena = arena;
  s->jobs = std::move(jobs);
  return VOPP_OK;
}

// Particle-steps of a batch (the leaf work dominates a plan's time).
double batch_steps(const std::vector<ServerReq> &batch) {
  double t = 0.0;
  for (const auto &r : batch) {
    const PlanShape &sh = r.job.shape;
    double lvl = (double)sh.N;
    for (int l = 1; l <= sh.D; ++l) { lvl *= sh.AW; t += lvl; }
  }
  return t;
}

// A free slot for a batch, or null.  Slot 0's stream has the device's highest priority:
// small batches take it first (their CTAs are then dispatched ahead of the queued CTAs of
// large plans already running on other slots), large batches take it last.
ServerSlot *pick_slot(vopp_server *srv, const std::vector<ServerReq> &batch) {
  const int n = (int)srv->slots.size();
  const bool small = batch_steps(batch) <= kSmallBatchSteps;
  for (int i = 0; i < n; ++i) {
    ServerSlot *s = srv->slots[small ? i : n - 1 - i];
    if (!s->busy) return s;
  }
  return nullptr;
}

// Completion state of a busy slot: 1 finished, 0 running, -1 failed.
int slot_state(ServerSlot *s) {
  const cudaError_t q = cudaEventQuery(s->done_ev);
  if (q == cudaSuccess) return 1;
  if (q == cudaErrorNotReady) return 0;
  cudaGetLastError();
  return -1;
}

// After the last batch finishes the worker keeps polling this long before it sleeps, so
// that a request arriving soon after starts without a thread wake-up (at a few thousand
// requests per second the worker then never sleeps: a serving process gives it a core).
constexpr double kSpinIdle = 2e-3;

void worker_main(vopp_server *srv) {
  cudaSetDevice(srv->c->device);
  double idle_since = now_s();
  std::vector<ServerSlot *> fin;
  std::vector<Harvest> hv;
  for (;;) {
    // finished slots: polled and gathered without the lock (slot state is this thread's)
    fin.clear();
    hv.clear();
    for (auto *s : srv->slots) {
      if (!s->busy.load() || s->launching.load()) continue;
      const int st = slot_state(s);
      if (st != 0) { fin.push_back(s); hv.push_back(gather(srv, s, st > 0)); }
    }
    int busy_now = 0;
    for (auto *s : srv->slots) busy_now += s->busy;
    if (fin.empty() && !srv->stop_flag.load()) {
      // nothing to post; nothing to start either (no request, or every slot busy): poll
      // again without the lock, in flight or within the idle polling window
      const size_t queued = srv->n_pending.load();
      if (busy_now > 0 && (queued == 0 || busy_now == (int)srv->slots.size())) {
        for (int k = 0; k < 8; ++k) cpu_relax();   // batches in flight: poll again soon
        idle_since = now_s();
        continue;
      }
      if (busy_now == 0 && queued == 0 && now_s() - idle_since < kSpinIdle) {
        std::this_thread::yield();
        continue;
      }
    }
    std::unique_lock<std::mutex> lock(srv->mu);
    bool posted = !fin.empty();
    for (size_t i = 0; i < fin.size(); ++i) post(srv, fin[i], hv[i]);
    for (;;) {
      if (srv->pending.empty() || (srv->paused && !srv->stop)) break;
      bool any_free = false;
      for (auto *q : srv->slots) any_free |= !q->busy;
      if (!any_free) break;
      const size_t refused_before = srv->completion_order.size();
      size_t bytes = 0;
      std::vector<ServerReq> batch = take_batch(srv, &bytes);
      posted |= srv->completion_order.size() != refused_before;
      if (batch.empty()) break;                 // the head waits for budget to free up
      ServerSlot *s = pick_slot(srv, batch);
      s->busy = true;
      lock.unlock();
      const int rc = launch_batch(srv, s, batch);
      lock.lock();
      if (rc != VOPP_OK) {                      // post the failure to every request
        srv->in_flight -= bytes;
        post_failure(srv, batch, rc);
        s->busy = false;
        posted = true;
        continue;
      }
      s->arena_bytes = bytes;                   // the reservation is released at post
      s->reqs = std::move(batch);
      srv->peak_in_flight = std::max(srv->peak_in_flight, srv->in_flight);
      srv->stats.batches += 1;
      srv->stats.batched_plans += s->reqs.size();
      srv->stats.max_batch_seen = std::max<uint64_t>(srv->stats.max_batch_seen, s->reqs.size());
    }
    if (posted) srv->cv_done.notify_all();
    int busy = 0;
    for (auto *s : srv->slots) busy += s->busy;
    if (srv->stop) {
      if (busy == 0 && srv->pending.empty()) break;
      // shutting down: wait (bounded) for the busy slots rather than polling at full rate
      lock.unlock();
      for (auto *s : srv->slots) {
        if (!s->busy || s->launching) continue;   // (a submitting thread's launch: next pass)
        int st = 0;
        for (int spins = 0; (st = slot_state(s)) == 0 && spins < 200000; ++spins)   // <= ~10 s
          std::this_thread::sleep_for(std::chrono::microseconds(50));
        Harvest h = gather(srv, s, st > 0);
        lock.lock();
        if (st == 0) srv->worker_error = VOPP_E_TIMEOUT;   // gave up on this batch
        post(srv, s, h);
        lock.unlock();
      }
      lock.lock();
      srv->cv_done.notify_all();
      continue;
    }
    if (busy || now_s() - idle_since < kSpinIdle) {
      // batches in flight, or only just idle: poll again, without holding the lock
      lock.unlock();
      std::this_thread::yield();
    } else {
      srv->cv_work.wait_for(lock, std::chrono::milliseconds(1), [&] {
        if (srv->stop || (!srv->pending.empty() && !srv->paused)) return true;
        for (auto *q : srv->slots)   // a batch a submitting thread launched
          if (q->busy && !q->launching) return true;
        return false;
      });
    }
    if (busy) idle_since = now_s();
  }
}

// Queue a request; or, when the server is idle (nothing queued, not paused, a slot free and
// the request within the budget), launch it at once as a batch of one on the calling thread,
// which saves the hand-off to the worker.  The worker then watches the slot as its own.
int submit_req(vopp_server *srv, ServerReq &&r, uint64_t *ticket) {
  std::vector<ServerReq> batch;
  ServerSlot *s = nullptr;
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    r.ticket = srv->next_ticket++;
    r.t_submit = now_s();
    *ticket = r.ticket;
    srv->stats.submitted += 1;
    if (srv->direct && !srv->stop && !srv->paused && srv->pending.empty() &&
        srv->in_flight + r.bytes <= srv->budget) {
      bytes = r.bytes;
      batch.push_back(std::move(r));
      s = pick_slot(srv, batch);
      if (s) {
        // launching first: the worker polls without the lock, reading busy and then
        // launching, so a slot it sees busy is one it also sees launching until the batch
        // is in place
        s->launching = true;
        s->busy = true;
        srv->in_flight += bytes;
      } else {
        r = std::move(batch.back());
        batch.clear();
      }
    }
    if (!s) {
      srv->pending.push_back(std::move(r));
      srv->n_pending.store(srv->pending.size());
    }
  }
  if (s) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != srv->c->device) cudaSetDevice(srv->c->device);
    const int rc = launch_batch(srv, s, batch);
    if (prev >= 0 && prev != srv->c->device) cudaSetDevice(prev);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (rc != VOPP_OK) {
      srv->in_flight -= bytes;
      post_failure(srv, batch, rc);
      s->busy = false;
      srv->cv_done.notify_all();
    } else {
      s->arena_bytes = bytes;
      s->reqs = std::move(batch);
      srv->peak_in_flight = std::max(srv->peak_in_flight, srv->in_flight);
      srv->stats.batches += 1;
      srv->stats.batched_plans += 1;
      srv->stats.max_batch_seen = std::max<uint64_t>(srv->stats.max_batch_seen, 1);
    }
    s->launching = false;
  }
  srv->cv_work.notify_one();
  return VOPP_OK;
}

}  // namespace

extern "C" {

int vopp_server_create(vopp_ctx *c, int32_t max_batch, int32_t n_slots, size_t hbm_budget_bytes,
                       vopp_server **out) {
  if (!c || !out || max_batch < 1 || n_slots < 1 || n_slots > 16)
    return fail(VOPP_E_INVALID, "bad server arguments");
  *out = nullptr;
  cudaSetDevice(c->device);
  vopp_server *srv = new (std::nothrow) vopp_server;
  if (!srv) return fail(VOPP_E_NOMEM, "server alloc");
  srv->c = c;
  srv->max_batch = max_batch;
  srv->use_graphs = c->use_graphs;
  srv->direct = c->server_direct != 0;
  srv->budget = hbm_budget_bytes ? hbm_budget_bytes : c->budget;
  for (int i = 0; i < n_slots; ++i) {
    ServerSlot *s = new (std::nothrow) ServerSlot;
    int prio_lo = 0, prio_hi = 0;   // numerically lower = higher priority
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (!s || cudaStreamCreateWithPriority(&s->slot.stream, cudaStreamNonBlocking,
                                           i == 0 ? prio_hi : prio_lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->done_ev, cudaEventDisableTiming) != cudaSuccess ||
        ensure_meta(s->slot, 1 << 20) != VOPP_OK) {
      if (s) {
        if (s->done_ev) cudaEventDestroy(s->done_ev);
        free_slot(s->slot);
        if (s->slot.stream) cudaStreamDestroy(s->slot.stream);
      }
      delete s;
      for (auto *q : srv->slots) {
        free_slot(q->slot);
        cudaEventDestroy(q->done_ev);
        cudaStreamDestroy(q->slot.stream);
        delete q;
      }
      delete srv;
      return fail(VOPP_E_NOMEM, "server slot");
    }
    srv->slots.push_back(s);
  }
  srv->worker = std::thread(worker_main, srv);
  *out = srv;
  return VOPP_OK;
}

void vopp_server_destroy(vopp_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
    srv->stop_flag.store(true);
  }
  srv->cv_work.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  for (auto *s : srv->slots) {
    if (s->kept) cudaFreeAsync(s->kept, s->slot.stream);
    cudaStreamSynchronize(s->slot.stream);
    s->graphs.release();
    free_slot(s->slot);
    cudaEventDestroy(s->done_ev);
    cudaStreamDestroy(s->slot.stream);
    delete s;
  }
  delete srv;
}

int vopp_submit(vopp_server *srv, const vopp_plan_request *req, uint64_t *ticket) {
  if (!srv || !req || !ticket) return fail(VOPP_E_INVALID, "NULL argument");
  if (!req->model || req->model->ctx != srv->c) return fail(VOPP_E_INVALID, "model of another context");
  ServerReq r;
  int rc = make_job(srv->c, req->model, req->root_states, req->root_weights, req->n_particles,
                    req->params, req->ptr_flags, r.job);
  if (rc) return rc;
  if (!(req->ptr_flags & VOPP_PTR_DEVICE)) {
    const size_t sb = root_words(r.job.shape.kind) * 4 * (size_t)r.job.shape.N;
    r.host_states.assign(static_cast<const char *>(req->root_states),
                         static_cast<const char *>(req->root_states) + sb);
    if (req->root_weights)
      r.host_weights.assign(reinterpret_cast<const char *>(req->root_weights),
                            reinterpret_cast<const char *>(req->root_weights) + 4 * (size_t)r.job.shape.N);
  }
  if (req->params.pi_bar) r.pi_bar.assign(req->params.pi_bar, req->params.pi_bar + req->model->A);
  r.bytes = r.job.lay.bytes + 256;
  return submit_req(srv, std::move(r), ticket);
}

int vopp_submit_agent(vopp_server *srv, vopp_agent *g, const vopp_plan_params *p, uint64_t *ticket) {
  if (!srv || !g || !p || !ticket) return fail(VOPP_E_INVALID, "NULL argument");
  if (g->model->ctx != srv->c) return fail(VOPP_E_INVALID, "agent of another context");
  ServerReq r;
  const void *states = g->blk;
  int rc = make_job(srv->c, g->model, states, nullptr, g->N, *p, VOPP_PTR_DEVICE, r.job);
  if (rc) return rc;
  r.job.log_weights = g->lw;
  if (g->reuse) attach_reuse(g, r.job);   // the worker allocates the kept tree's memory
  if (p->pi_bar) r.pi_bar.assign(p->pi_bar, p->pi_bar + g->model->A);
  r.bytes = r.job.lay.bytes + 256;
  return submit_req(srv, std::move(r), ticket);
}

static int take_done(vopp_server *srv, uint64_t ticket, vopp_plan_result *out, double *latency) {
  auto it = srv->done.find(ticket);
  if (it == srv->done.end()) return VOPP_E_BUSY;
  const Done d = it->second;
  srv->done.erase(it);
  if (out) *out = d.res;
  if (latency) *latency = d.t_done - d.t_submit;
  if (d.status) return fail(d.status, "request failed");
  return VOPP_OK;
}

int vopp_poll(vopp_server *srv, uint64_t ticket, vopp_plan_result *out, double *latency_s) {
  if (!srv) return fail(VOPP_E_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  return take_done(srv, ticket, out, latency_s);
}

int vopp_wait(vopp_server *srv, uint64_t ticket, double timeout_s, vopp_plan_result *out,
              double *latency_s) {
  if (!srv) return fail(VOPP_E_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lock(srv->mu);
  auto ready = [&] { return srv->done.count(ticket) > 0; };
  // a zero timeout only looks (a timed wait would still sleep for the kernel's timer slack)
  const bool ok = timeout_s > 0.0
                      ? srv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready)
                      : ready();
  if (!ok) return fail(VOPP_E_TIMEOUT, "ticket not completed within the timeout");
  return take_done(srv, ticket, out, latency_s);
}

int vopp_wait_any(vopp_server *srv, double timeout_s, uint64_t *ticket, vopp_plan_result *out,
                  double *latency_s) {
  if (!srv || !ticket) return fail(VOPP_E_INVALID, "NULL argument");
  auto ready = [&] {   // (lock held)
    while (!srv->completion_order.empty() && !srv->done.count(srv->completion_order.front()))
      srv->completion_order.pop_front();   // already taken by vopp_poll / vopp_wait
    srv->n_order.store(srv->completion_order.size());
    return !srv->completion_order.empty();
  };
  auto take_front = [&] {   // (lock held, ready() true)
    *ticket = srv->completion_order.front();
    srv->completion_order.pop_front();
    srv->n_order.store(srv->completion_order.size());
    return take_done(srv, *ticket, out, latency_s);
  };
  // a short timeout spins on the completion count (no lock, no sleep) until a plan has
  // finished or the time is up; entries of tickets already taken by vopp_poll / vopp_wait
  // are dropped under the lock and the spin goes on
  if (timeout_s > 0.0 && timeout_s <= kSpinWaitMax) {
    const double t_end = now_s() + timeout_s;
    for (;;) {
      while (srv->n_order.load() == 0 && now_s() < t_end)
        for (int k = 0; k < 4; ++k) cpu_relax();
      if (srv->n_order.load() == 0) return fail(VOPP_E_TIMEOUT, "no plan completed within the timeout");
      std::unique_lock<std::mutex> lock(srv->mu);
      if (ready()) return take_front();
      if (now_s() >= t_end) return fail(VOPP_E_TIMEOUT, "no plan completed within the timeout");
    }
  }
  // a zero-timeout poll with nothing finished answers without the lock, so that a caller
  // polling in a loop never holds up the worker
  if (!(timeout_s > 0.0) && srv->n_order.load() == 0)
    return fail(VOPP_E_TIMEOUT, "no plan completed within the timeout");
  std::unique_lock<std::mutex> lock(srv->mu);
  const bool ok = timeout_s > 0.0
                      ? srv->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), ready)
                      : ready();   // a zero timeout only looks
  if (!ok) return fail(VOPP_E_TIMEOUT, "no plan completed within the timeout");
  return take_front();
}

int vopp_server_set_paused(vopp_server *srv, int paused) {
  if (!srv) return fail(VOPP_E_INVALID, "server is NULL");
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->paused = paused != 0;
  }
  srv->cv_work.notify_one();
  return VOPP_OK;
}

int vopp_server_get_stats(vopp_server *srv, vopp_server_stats *out) {
  if (!srv || !out) return fail(VOPP_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(srv->mu);
  *out = srv->stats;
  out->pending = srv->pending.size();
  out->in_flight_bytes = srv->in_flight;
  out->peak_in_flight_bytes = srv->peak_in_flight;
  return VOPP_OK;
}

}  // extern "C"

