// vopp_internal.h -- declarations shared by the kernels and the host-side C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "vopp.h"
#include "vopp_device.cuh"

namespace vopp {

// NVTX range for the lifetime of a scope: a profiler (Nsight Systems, ncu's NVTX filters)
// shows each plan, batch, belief update and kernel launch as a named range; without a tool
// attached a push/pop costs a branch.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct BeliefOut {
  int status;       // 0 ok, 1 degenerate (every particle has zero likelihood)
  int resampled;
  double ess;
};

struct BeliefArgs {
  int kind, N, action;
  uint32_t key0, key1;
  unsigned long long t;        // agent time step (Philox node word)
  float *x, *y, *lw;           // current belief (NAV2D x, y)
  int *s;                      // current belief (GRID / TOY2)
  float *tx, *ty, *tlw;        // propagated particles (scratch)
  int *ts;
  float *pf, *tpf;             // CROWD people [12][N] (current, propagated)
  double *cdf;                 // [N] scratch
  int *anc;                    // [N] ancestors of the update
  float obs_f[2];
  int obs_i;
  const DevModel *model;
  BeliefOut *out;
};

struct EnvOut {
  float obs[2];     // NAV2D observation
  int obs_i;        // GRID / TOY2 observation
  float reward;
  int terminal;
};

// One step of the closed loop's true state (a single particle on the device).
struct EnvArgs {
  int kind, action;
  uint32_t key0, key1;
  unsigned long long t;        // environment time step (Philox node word)
  float *xy;                   // NAV2D / CROWD robot (x, y)
  int *s;                      // GRID / TOY2 state, CROWD flags
  float *pf;                   // CROWD people (x, y) x 6
  const DevModel *model;
  EnvOut *out;
};

// CROWD leaf CTAs have five warps whatever the leaf-threads option: the model's A W = 5 W
// branches then divide evenly among them.
constexpr int kCrowdLeafThreads = 160;

// Dynamic shared memory a leaf CTA may use (B300: 227 KB per block, kept below it).
constexpr size_t kLeafSmemLimit = 200 * 1024;
size_t leaf_smem_bytes(int kind, int N, int AW);
size_t expand_smem_bytes(int N);
// an expansion stage whose level-0 items prepare the root themselves (PlanDesc::root_fused)
size_t expand_fused_smem_bytes(int kind, int N);
cudaError_t launch_root_prep(const PlanDesc *d, const StageTable &st, cudaStream_t s);
cudaError_t init_kernel_attributes();
// wide: the stage has at most one CTA per SM (wider CTAs, fewer particles per thread)
cudaError_t launch_expand(const PlanDesc *d, const StageTable &st, long long total, size_t smem,
                          long long grid, bool wide, cudaStream_t s);
// kind selects the model's leaf kernel (kNav, kGrid, kToy)
// Vectorised expansion (NAV2D, GRID, TOY2): vw particles per lane unit (4, 2 or 1, dividing
// every plan's N); one child per warp, kExpandVecChildrenPerCta children per CTA.
#ifndef VOPP_EXPAND_VEC_THREADS
#define VOPP_EXPAND_VEC_THREADS 128
#endif
constexpr int kExpandVecChildrenPerCta = VOPP_EXPAND_VEC_THREADS / 32;
// Levels (counted in the full tree of their Philox keys) narrower than this expand one CTA
// per child instead.
constexpr long long kExpandVecMinChildren = 512;
cudaError_t launch_expand_vec(int kind, int vw, const PlanDesc *d, const StageTable &st,
                              long long total, long long grid, cudaStream_t s);
cudaError_t launch_leaf(int kind, const PlanDesc *d, const StageTable &st, long long total,
                        size_t smem, int threads, long long grid, cudaStream_t s);
cudaError_t leaf_occupancy(int kind, int threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_belief(const BeliefArgs &B, cudaStream_t s);
// n updates, args in device memory (one CTA each, the same arithmetic as launch_belief)
cudaError_t launch_belief_batch(const BeliefArgs *d_args, int n, cudaStream_t s);
cudaError_t launch_env(const EnvArgs &E, cudaStream_t s);

// A batch of device-to-device copies (src null: zero dst) in one launch: the arrays a plan
// that continues a kept subtree takes from it, or an adopted subtree's nodes.  Every
// address and size is a multiple of 4 bytes.
constexpr int kMaxCopyOps = 48;
struct CopyList {
  int n;
  void *dst[kMaxCopyOps];
  const void *src[kMaxCopyOps];
  unsigned long long bytes[kMaxCopyOps];
};
cudaError_t launch_copy_list(const CopyList &L, cudaStream_t s);
// The same from a descriptor table in device memory (n entries; `most` = the largest size).
struct CopyDesc {
  void *dst;
  const void *src;
  unsigned long long bytes;
};
cudaError_t launch_copy_table(const CopyDesc *table, int n, unsigned long long most, cudaStream_t s);
// Root preparation with the copies of continued subtrees in the same launch: one CTA per
// plan of the stage (a continued plan's CTA first makes its own level-0 copies), then CTAs
// for slices of table entries 0 .. n_rest - 1 (the other levels' copies; `most`: the largest).
cudaError_t launch_root_prep_copy(const PlanDesc *d, const StageTable &st, const CopyDesc *table,
                                  int n_rest, unsigned long long most, cudaStream_t s);

}  // namespace vopp

struct vopp_model;
struct vopp_ctx;
namespace vopp {
const DevModel *model_device_tables(const vopp_model *m);
int model_kind(const vopp_model *m);
int model_device(const vopp_model *m);
const vopp_model_desc &model_desc(const vopp_model *m);
vopp_ctx *model_ctx(const vopp_model *m);
cudaStream_t model_stream(const vopp_model *m);
cudaStream_t ctx_stream(const vopp_ctx *c);
int set_error(int code, const char *msg);   // records the thread-local message, returns code

// Episode mode (vopp_episodes.cu): buffers of a context's last episode-mode plan.
struct EpisodeStore;
EpisodeStore *&ctx_episode_store(vopp_ctx *c);
void free_episode_store(EpisodeStore *s);
struct EpisodeInputs {
  const void *states;         // NAV2D float[2N] (x then y), GRID / TOY2 int32[N]
  const float *weights;       // linear weights or null (uniform)
  const float *log_weights;   // device log weights (agents) or null
  int N;
  uint32_t ptr_flags;
};
int run_plan_episodes(vopp_model *m, const EpisodeInputs &in, const vopp_episode_params &p,
                      double budget_s, vopp_plan_result *out, int32_t *depth_reached,
                      int32_t *n_nodes);
int episode_tree_read(vopp_ctx *c, int32_t field, uint64_t offset, uint64_t count, void *dst);

}  // namespace vopp
