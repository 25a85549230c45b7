/*
 * vopp.h -- C ABI of libvopp, a B300 (sm_103a) implementation of the data-parallel hot path
 * of VOPP, the Vectorized Online POMDP Planner ("Vectorized Online POMDP Planning",
 * arXiv 2510.27191).
 *
 * What one plan computes (paper Sec. III):
 *   - Alg. 1: sample the root belief (here: the caller's weighted particle set), run one
 *     search episode, back it up, return argmax_a Psi(root, a).
 *   - Alg. 2 (forward search), full-width form: every belief node expands every action a and
 *     W observation branches per action.  Each branch steps ALL N particles of its parent
 *     through the generative model G(s,a) -> (s', o, r) (Sec. III-B), draws one
 *     observation o_k from a representative particle (or enumerates o_k = k), and reweights
 *     the particles by Z(o_k | s', a).  Leaves (depth D) take the weighted mean of a
 *     state-based heuristic (Alg. 2 ValueHeuristic).
 *   - Alg. 3 (backup), closed form of one Eq. 3 preference update from the reference
 *     policy pibar: Q(b,a) = (1/W) sum_k rbar_k + gamma * sum_k omega_k V_k / sum_k omega_k,
 *     V(b) = eta * log sum_a pibar(a|b) exp(Q(b,a)/eta)  (Eq. 1; eta is the temperature,
 *     the paper's eta is 1/eta).
 *   - Sec. III-B: the belief update tau(b,a,o) is a sequential importance resampling filter.
 *
 * Conventions for every entry point:
 *   - Every call returns an int status (VOPP_OK or a negative VOPP_E_* code); no C++
 *     exception crosses the ABI.  vopp_last_error() gives a thread-local message for the most
 *     recent failure on the calling thread.
 *   - Caller buffers are only read or written during the call; the library keeps no pointer
 *     to them after it returns.  Pointers are host pointers unless the call takes
 *     ptr_flags with VOPP_PTR_DEVICE set, in which case they are device pointers on the
 *     context's device (e.g. a torch tensor's data_ptr()).
 *   - The library owns all device memory it allocates (per-context arena, models, agents);
 *     destroy functions release it.
 *   - All device work is issued on the context's CUDA stream (given at creation; 0 = the
 *     legacy default stream).  Blocking calls synchronise that stream before returning.
 *   - Kernels never trap: device-side failures (zero-mass beliefs, exhausted waits) are
 *     reported through a device status word that the host reads back.
 *   - A context, and every model and agent created from it, must be used by one host thread
 *     at a time.
 */
#ifndef VOPP_H
#define VOPP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VOPP_API __attribute__((visibility("default")))
#else
#define VOPP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------------- */
#define VOPP_OK 0
#define VOPP_E_INVALID (-1)    /* an argument is out of range or a pointer is NULL        */
#define VOPP_E_NOMEM (-2)      /* a device or host allocation failed                      */
#define VOPP_E_BUDGET (-3)     /* the plan's predicted footprint exceeds the HBM budget   */
#define VOPP_E_CUDA (-4)       /* a CUDA runtime call failed (message in vopp_last_error) */
#define VOPP_E_TIMEOUT (-5)    /* a bounded device-side wait gave up                      */
#define VOPP_E_DEGENERATE (-6) /* the (root or updated) belief has zero total weight      */
#define VOPP_E_BUSY (-7)       /* the ticket's plan has not completed yet                 */

/* ---- model kinds, branch modes, reference policies ----------------------------------- */
#define VOPP_NAV2D 0 /* continuous 2-D navigation, state (x,y) in [0,10]^2, 4 actions     */
#define VOPP_GRID 1  /* 11x11 grid sensing, packed int32 state, 13 actions, obs {0,1,2}  */
#define VOPP_TOY2 2  /* 2 states, 2 actions, 2 observations (test model)                  */
#define VOPP_CROWD 3 /* crowd navigation shaped like the paper's CrowdNav (Sec. IV): robot in
                        a 50 x 40 m hall with its 6 nearest people, each curious or shy
                        (hidden); 5 actions (NORTH, EAST, SOUTH, WEST, YELL); 64 observations
                        (per person: came closer, each bit flipped with probability 0.1);
                        gamma 0.97 in the paper.  Particle layout: 15 rows of N 32-bit words
                        -- robot x, robot y, people x0 y0 ... x5 y5 (float32), then int32
                        flags (bits 0-5 traits, 1 = curious; 8-13 "came closer"; 16
                        terminal).  A person's "came closer" bit is decided from its
                        displacement d before the hall's walls clamp the new position:
                        d.(d + 2(p - r)) < 0, with p its old position and r the robot's new
                        one.  Away from the walls this is exactly |p + d - r| < |p - r|; for
                        a person a wall stops, the bit describes the attempted move, not the
                        clamped one.  ENUMERATE branches and the distance-softmax policy are
                        not available. */

#define VOPP_BRANCH_SAMPLE 0    /* o_k drawn from a uniformly chosen representative      */
#define VOPP_BRANCH_ENUMERATE 1 /* branch k is observation k (discrete models, W >= |O|) */

#define VOPP_PI_UNIFORM 0  /* pibar(a|b) = 1/A                                            */
#define VOPP_PI_FIXED 1    /* pibar(a|b) = pi_fixed[a] / sum pi_fixed                       */
#define VOPP_PI_NAV_DIST 2 /* pibar(a|b) ~ exp(-|clamp(mu_b + delta_a)| / pi_temp), NAV2D   */

#define VOPP_PTR_DEVICE 1u /* ptr_flags bit: the state/weight pointers are device pointers */

/* result flags */
#define VOPP_FLAG_DEGENERATE_BRANCH 1u /* some action had sum_k omega_k = 0 (future := 0) */
#define VOPP_FLAG_FP64_ROOT 2u         /* the root backup ran in FP64                     */
#define VOPP_FLAG_REUSED 4u            /* the plan continued a kept subtree (agents with
                                          subtree reuse, vopp_agent_set_reuse)             */

/* tree detail kept on the device after a plan (vopp_ctx_set_tree_detail) */
#define VOPP_TREE_MINIMAL 0 /* only what the backup needs                                 */
#define VOPP_TREE_FULL 1    /* also leaf-level branch stats, representatives, observations */

/* tree fields readable with vopp_tree_read (per level, indexed by node or child) */
#define VOPP_FIELD_V 0      /* float  V[node]               levels 0..D (D: leaves, FULL)  */
#define VOPP_FIELD_Q 1      /* float  Q[node][A]            levels 0..D-1                  */
#define VOPP_FIELD_RBAR 2   /* float  rbar[child]           levels 1..D (D only if FULL)   */
#define VOPP_FIELD_LOMEGA 3 /* float  log omega[child]      levels 1..D (D only if FULL)   */
#define VOPP_FIELD_REP 4    /* int32  representative j      levels 1..D (FULL)             */
#define VOPP_FIELD_OBS 5    /* float  observation[child][2] levels 1..D (FULL)             */
#define VOPP_FIELD_PX 6     /* float  NAV2D x[node][N]      materialised levels            */
#define VOPP_FIELD_PY 7     /* float  NAV2D y[node][N]      materialised levels            */
#define VOPP_FIELD_PS 8     /* int32  GRID/TOY2 s, CROWD flags [node][N], materialised     */
#define VOPP_FIELD_PLW 9    /* float  log weight[node][N]   materialised levels            */
#define VOPP_FIELD_MU 10    /* float  weighted mean particle [node][2] (VOPP_PI_NAV_DIST) */
#define VOPP_FIELD_PSI 11   /* float  Psi[node][A] persistent preferences, levels 0..D-1,
                               after vopp_plan_anytime / vopp_agent_plan_anytime only        */
#define VOPP_FIELD_PF 12    /* float  CROWD people [node][12][N] (rows x0 y0 .. x5 y5),
                               materialised levels (robot in PX / PY, flags in PS)           */

#define VOPP_MAX_ACTIONS 16
#define VOPP_MAX_DEPTH 8
#define VOPP_MAX_PARTICLES 65536 /* agents / belief updates; a plan's leaf kernel stages one
                                     node's particles in shared memory, which bounds N to
                                     12,600 (NAV2D) or 16,800 (GRID, TOY2) at A*W <= 64 */

typedef struct vopp_ctx vopp_ctx;
typedef struct vopp_model vopp_model;
typedef struct vopp_agent vopp_agent;

/* Model description.  The POMDP 8-tuple of Sec. II-A fixed by kind; layout fields apply
 * to VOPP_GRID (rock cells, all distinct, none on the start cell (0,5)). */
typedef struct {
  int32_t kind;        /* VOPP_NAV2D | VOPP_GRID | VOPP_TOY2 | VOPP_CROWD                  */
  int32_t branch_mode; /* VOPP_BRANCH_SAMPLE | VOPP_BRANCH_ENUMERATE                      */
  int32_t pi_mode;     /* VOPP_PI_UNIFORM | VOPP_PI_FIXED | VOPP_PI_NAV_DIST                */
  int32_t h_zero;      /* 1: leaf heuristic forced to 0                                    */
  float pi_temp;       /* temperature of VOPP_PI_NAV_DIST                                  */
  float pi_fixed[VOPP_MAX_ACTIONS]; /* VOPP_PI_FIXED weights (>= 0, positive sum)          */
  int32_t rock_x[8], rock_y[8];     /* VOPP_GRID rock cells                                */
} vopp_model_desc;

/* Result of one plan (Alg. 1 action selection and the root's backed-up values). */
typedef struct {
  int32_t action;                    /* argmax_a Q(root,a) + eta log pibar(a|root), lowest
                                        index on ties                                      */
  uint32_t flags;                    /* VOPP_FLAG_*                                        */
  double v_root;                     /* V(root)                                            */
  double q[VOPP_MAX_ACTIONS];        /* Q(root, a), a < A                                  */
  double policy[VOPP_MAX_ACTIONS];   /* pi*(a) = pibar(a) exp((Q_a - V)/eta)               */
  uint64_t particle_steps;           /* sum_{l=1..D} (A W)^l N generative-model steps      */
  uint64_t nodes;                    /* belief nodes in the tree, root included            */
  uint32_t degenerate_actions;       /* actions whose branch weights all vanished          */
  uint32_t reused_levels;            /* with VOPP_FLAG_REUSED: materialised levels below the
                                        root copied from the kept subtree instead of
                                        expanded again (else 0)                            */
} vopp_plan_result;

/* Per-plan parameters (used by agents, batches and the serving queue). */
typedef struct {
  int32_t depth;          /* D >= 0 action levels                                          */
  int32_t width;          /* W >= 1 observation branches per action                        */
  float eta;              /* temperature > 0                                               */
  float gamma;            /* discount in (0,1)                                             */
  uint64_t seed;          /* Philox key of the plan                                        */
  const float *pi_bar;    /* [A] host weights overriding the model's reference policy, or NULL */
} vopp_plan_params;

/* One plan of a batch: root particles (host or device per ptr_flags) plus parameters. */
typedef struct {
  vopp_model *model;
  const void *root_states;  /* NAV2D: float[2N] (x[0..N-1] then y[0..N-1]); GRID/TOY2: int32[N];
                               CROWD: 15 rows of N words (see VOPP_CROWD)                   */
  const float *root_weights;/* [N] or NULL for uniform                                    */
  int32_t n_particles;
  uint32_t ptr_flags;
  vopp_plan_params params;
} vopp_plan_request;

/* ---- context ------------------------------------------------------------------------- */
/* Create a context on CUDA device `device`, issuing work on `cuda_stream` (a cudaStream_t
 * cast to an integer; 0 = legacy default stream).  hbm_budget_bytes caps the device arena
 * the context may allocate (0 = 80% of the device's free memory at creation). */
VOPP_API int vopp_ctx_create(int device, size_t hbm_budget_bytes, uintptr_t cuda_stream, vopp_ctx **out);
VOPP_API void vopp_ctx_destroy(vopp_ctx *ctx);
/* VOPP_TREE_MINIMAL (default) or VOPP_TREE_FULL. */
VOPP_API int vopp_ctx_set_tree_detail(vopp_ctx *ctx, int detail);
/* Tuning options (vopp_ctx_set_option):
 *   VOPP_OPT_LEAF_GEN        1 (default): the leaf kernel builds level D-1 in shared memory
 *                            from level D-2; 0: level D-1 is materialised in HBM first
 *   VOPP_OPT_LEAF_THREADS    threads per leaf CTA, multiple of 32 in [32, 256] (default 128;
 *                            CROWD leaf CTAs always have 160: five warps for its 5 W branches)
 *   VOPP_OPT_GRID_CAP        maximum CTAs of an expansion / leaf launch (grid-stride beyond)
 * Results do not depend on any option. */
#define VOPP_OPT_LEAF_GEN 1
#define VOPP_OPT_LEAF_THREADS 2
#define VOPP_OPT_GRID_CAP 3
#define VOPP_OPT_PERSISTENT 5   /* 1: leaf CTAs fill every SM once and pull work items from a
                                   counter (largest items first); 0: one CTA per item; 2
                                   (default): per model, persistent for GRID and TOY2 (the
                                   grid leaf's many short items), one CTA per item for NAV2D
                                   and CROWD; other values: VOPP_E_INVALID */
#define VOPP_OPT_FP64_ROOT 6    /* 1: back the root up in FP64 (VOPP_FLAG_FP64_ROOT); 0 (default):
                                   FP32 with compensated sums, within the 1e-4 tolerance */
#define VOPP_OPT_GRAPHS 7       /* 1: vopp_plan / vopp_plan_batch capture their launch sequence in
                                   a CUDA graph and replay it while the batch shape, buffers and
                                   options repeat (not while per-kernel timing is on, and not for
                                   batches that keep or continue agents' trees) */
#define VOPP_OPT_REUSE_COPY 8   /* 1 (default): a plan that continues a kept subtree copies its
                                   materialised levels; 0: it expands them again under the same
                                   keys (the same result; for checking the copies) */
#define VOPP_OPT_SERVER_DIRECT 9 /* 1: a server created while the option is on lets
                                   a submitting thread that finds it idle (nothing queued, a
                                   slot free, the request within the budget) launch the request
                                   itself, as a batch of one, instead of handing it to the
                                   worker (the submit call then returns after the launch,
                                   without waiting for the device); 0 (default): the worker
                                   launches every batch (for a caller that submits and
                                   collects on one thread the cheaper submit measured better:
                                   the launch no longer delays its noticing other plans'
                                   completions) */
VOPP_API int vopp_ctx_set_option(vopp_ctx *ctx, int32_t option, int64_t value);
/* Enable (1) / disable (0) per-kernel CUDA-event timing on the context's stream. */
VOPP_API int vopp_ctx_set_timing(vopp_ctx *ctx, int enable);
/* Per-kernel-family accumulated device time (ms) and launch counts since the last reset:
 * root_prep, expand, leaf, belief, then expand_to_l1 .. expand_to_l8 (the expansion
 * launches that wrote that level, also counted under expand).
 * names[i] receives a static string; arrays hold at least *n entries on input; *n is set
 * to the number of families written. */
VOPP_API int vopp_ctx_kernel_times(vopp_ctx *ctx, const char **names, double *ms, uint64_t *launches,
                          int *n);
VOPP_API int vopp_ctx_reset_kernel_times(vopp_ctx *ctx);
/* Host->device and device->host bytes the context copied, and kernels it launched, since
 * the last vopp_ctx_reset_kernel_times (each pointer may be NULL). */
VOPP_API int vopp_ctx_counters(vopp_ctx *ctx, uint64_t *h2d_bytes, uint64_t *d2h_bytes,
                               uint64_t *launches);
/* Device bytes a plan of this shape needs in the arena (for admission control). */
VOPP_API int vopp_plan_footprint(const vopp_model *model, int32_t n_particles, int32_t depth,
                        int32_t width, size_t *bytes);

/* ---- models -------------------------------------------------------------------------- */
/* Validate a model description and upload its constant tables. */
VOPP_API int vopp_create_model(vopp_ctx *ctx, const vopp_model_desc *desc, vopp_model **out);
VOPP_API void vopp_model_destroy(vopp_model *model);
/* Number of actions A of the model's kind (4, 13 or 2); negative status on NULL. */
VOPP_API int vopp_model_num_actions(const vopp_model *model);

/* ---- one plan (Alg. 1 with one full-width search and one backup) ---------------------- */
/* root_states: NAV2D float[2N] (x then y), GRID/TOY2 int32[N], CROWD 15 rows of N words
 * (robot x, y, 12 people coordinates, int32 flags); root_weights: [N] or NULL.
 * A GRID state is packed: bits 0-7 rock bits, 8-11 x in 0..11 (11 = exited), 12-15 y in
 * 0..10, bit 16 terminal, bits 17-31 clear.  Host states outside that are rejected
 * (VOPP_E_INVALID, also by vopp_agent_create and vopp_env_create); a device buffer is not
 * read on the host, and its out-of-range fields are clamped on load.
 * Weights must be >= 0; particles that are terminal at the root get weight 0; zero total
 * weight returns VOPP_E_DEGENERATE.  pi_bar: [A] host weights or NULL (model's policy).
 * Errors: VOPP_E_INVALID for depth < 0 or > VOPP_MAX_DEPTH, width < 1, N < 1 or
 * > VOPP_MAX_PARTICLES, eta <= 0, gamma outside (0,1), invalid pi_bar; VOPP_E_BUDGET when
 * the footprint exceeds the budget.  Depth 0 returns V = weighted mean heuristic, every
 * Q equal to it and the action argmax pibar. */
VOPP_API int vopp_plan(vopp_model *model, const void *root_states, const float *root_weights,
              int32_t n_particles, int32_t depth, int32_t width, float eta, float gamma,
              const float *pi_bar, uint64_t seed, uint32_t ptr_flags, vopp_plan_result *out);

/* vopp_plan in two halves, for callers that overlap host work with the plan or time it on
 * the device: vopp_plan_submit checks the arguments and enqueues the whole plan on the
 * context's stream (same arguments and errors as vopp_plan; host inputs are copied before it
 * returns, device inputs must stay valid until vopp_plan_finish); vopp_plan_finish waits for
 * it and fills *out exactly as vopp_plan would.  One submitted plan per context: while it is
 * pending, vopp_plan_submit, every plan call, tree reads, autotuning and option changes on
 * the context return VOPP_E_BUSY; vopp_plan_finish with nothing pending returns
 * VOPP_E_INVALID; vopp_ctx_destroy waits for a pending plan. */
VOPP_API int vopp_plan_submit(vopp_model *model, const void *root_states, const float *root_weights,
                              int32_t n_particles, int32_t depth, int32_t width, float eta,
                              float gamma, const float *pi_bar, uint64_t seed, uint32_t ptr_flags);
VOPP_API int vopp_plan_finish(vopp_ctx *ctx, vopp_plan_result *out);
/* The context a model was created in (NULL for NULL). */
VOPP_API vopp_ctx *vopp_model_ctx(const vopp_model *model);

/* ---- anytime plan (Alg. 1 planning loop with iterative deepening, Eq. 3) --------------- */
/* Iterations k = 1, 2, ..., params->depth: iteration k searches the full-width tree of
 * depth k with the plan's seed -- so a node has the same particles in every iteration --
 * and backs it up with the preference update of Eq. 3 on preferences Psi(n, .) that persist
 * across iterations (Alg. 3: V_curr = eta log sum_a exp(Psi/eta); Psi <- Psi - V_curr + Q;
 * V = eta log sum_a exp(Psi/eta)); the nodes of level k-1 are new in iteration k and start
 * from Psi_0 = eta log pibar.  Iteration 1 equals vopp_plan at depth 1.  A further
 * iteration starts while the wall time since the call began is below budget_s (<= 0: no
 * time limit, run to params->depth); the last iteration may overrun the budget.
 * out: the last iteration's root Q, V = [L Psi](root), policy softmax(Psi/eta) and action
 * argmax Psi (lowest index on ties); particle_steps counts the steps actually simulated
 * (each iteration adds one materialised level, rebuilds the leaf kernel's node level and
 * expands the leaves).  depth_reached (may be NULL) receives the last iteration's depth.
 * Arguments, layouts, ownership and errors as vopp_plan; params->depth >= 1. */
VOPP_API int vopp_plan_anytime(vopp_model *model, const void *root_states, const float *root_weights,
                               int32_t n_particles, const vopp_plan_params *params, double budget_s,
                               uint32_t ptr_flags, vopp_plan_result *out, int32_t *depth_reached);

/* ---- episode mode (Alg. 1-3 as printed) ---------------------------------------------- */
/* Planning iterations k = 1, 2, ..., max_depth (D_max = k): sample `episodes` root states
 * from the belief (Philox purpose 7; episode e, iteration k), run every episode to depth k
 * -- action a ~ softmax(Psi(b,.)/eta) (purpose 8), G (transition purpose 9, observation
 * purpose 10, depth d as the level word), reward and visit added to action node (b, a), the
 * episode ends at a terminal state, else moves to the child belief of its observation,
 * created on first visit (a continuous NAV2D observation always creates one) -- then
 * aggregate the leaf heuristics and back up (Alg. 3) for d = k..1: W(b,a) = sum over the
 * children of visits x V (normaliser: the action's own visits, so terminated episodes add no
 * future value), Q = C/N + gamma W/N (0 for an action without visits), and every belief at
 * depth d-1: V_curr = eta log sum exp(Psi/eta), Psi <- Psi - V_curr + Q, V = L Psi.  A new
 * belief starts from Psi_0 = eta log pibar (uniform or fixed policy; the distance softmax
 * needs per-node particle sets and is refused with VOPP_E_INVALID).  Another iteration
 * starts while the wall time is below budget_s (<= 0: none).  Node ids follow creation
 * order (iteration, depth, episode); the tree lives until the next episode-mode plan on the
 * context (vopp_episode_tree_read).  out: action argmax Psi(root), v_root = V(root), q =
 * the root's last Q, policy softmax(Psi(root)/eta), particle_steps = generative-model calls,
 * nodes = beliefs.  Errors: VOPP_E_INVALID (arguments), VOPP_E_NOMEM (device buffers, or
 * more beliefs than max_nodes), VOPP_E_DEGENERATE (root weights sum to 0). */
typedef struct {
  int32_t episodes;    /* M, episodes per planning iteration, 1 .. 2^24                   */
  int32_t max_depth;   /* iterations = maximum depth, 1 .. VOPP_MAX_DEPTH                 */
  float eta;           /* temperature (> 0)                                               */
  float gamma;         /* discount in (0,1)                                               */
  uint64_t seed;       /* Philox key                                                      */
  int32_t max_nodes;   /* belief capacity; 0: M * D * (D + 1) / 2 + 1 (always enough)     */
} vopp_episode_params;
VOPP_API int vopp_plan_episodes(vopp_model *model, const void *root_states, const float *root_weights,
                                int32_t n_particles, const vopp_episode_params *params, double budget_s,
                                uint32_t ptr_flags, vopp_plan_result *out, int32_t *depth_reached,
                                int32_t *n_nodes);
/* Fields of the last episode-mode tree (vopp_episode_tree_read), indexed by belief id. */
#define VOPP_EP_PARENT 0   /* int32  parent action node b*A + a, -1 at the root              */
#define VOPP_EP_DEPTH 1    /* int32  depth                                                   */
#define VOPP_EP_PSI 2      /* double Psi[node][A]                                            */
#define VOPP_EP_V 3        /* double V[node]                                                 */
#define VOPP_EP_REWARD 4   /* double C[node][A], reward sum of the action node               */
#define VOPP_EP_VISITS 5   /* uint64 N[node][A], visits of the action node                   */
/* Copy `count` elements from element `offset` of a field of the context's last episode-mode
 * tree to host memory dst. */
VOPP_API int vopp_episode_tree_read(vopp_ctx *ctx, int32_t field, uint64_t offset, uint64_t count,
                                    void *dst);

/* Copy `count` elements of a tree field of the most recent plan on this context, starting
 * at element `offset` of that level's array, into dst (host, or device with ptr_flags).
 * Valid until the next plan on the context. */
VOPP_API int vopp_tree_read(vopp_ctx *ctx, int32_t field, int32_t level, uint64_t offset, uint64_t count,
                   void *dst, uint32_t ptr_flags);

/* Same as vopp_tree_read for plan `plan` (0-based) of the most recent batch. */
VOPP_API int vopp_tree_read_plan(vopp_ctx *ctx, int32_t plan, int32_t field, int32_t level, uint64_t offset,
                        uint64_t count, void *dst, uint32_t ptr_flags);

/* The GRID sense-outcome thresholds floor(acc(d2) 2^32), d2 = 0..n-1 (n <= 256), exactly
 * as uploaded by vopp_create_model: a sampled outcome is correct iff a Philox word is below
 * thr[d2].  Host-only; needs no device. */
VOPP_API int vopp_grid_thresholds(uint64_t *thr, int32_t n);

/* ---- agents: device-resident beliefs with the SIR update (Sec. III-B) ---------------- */
/* An agent holds n weighted particles (states as for vopp_plan's root, weights linear or
 * NULL = uniform, host or device per ptr_flags) on the device, with its own Philox key
 * (seed) and time step for its belief updates.  Its device memory comes from the device's
 * stream-ordered pool on the context's stream, so creating or destroying an agent does not
 * synchronise the device (a serving loop keeps running while agents come and go); do not
 * destroy an agent while a request on it is outstanding. */
VOPP_API int vopp_agent_create(vopp_model *model, const void *states, const float *weights, int32_t n,
                      uint64_t seed, uint32_t ptr_flags, vopp_agent **out);
VOPP_API int vopp_agent_plan(vopp_agent *agent, const vopp_plan_params *params, vopp_plan_result *out);
/* vopp_plan_episodes from the agent's particles and log weights. */
VOPP_API int vopp_agent_plan_episodes(vopp_agent *agent, const vopp_episode_params *params, double budget_s,
                                      vopp_plan_result *out, int32_t *depth_reached, int32_t *n_nodes);
/* vopp_plan_anytime from the agent's particles. */
VOPP_API int vopp_agent_plan_anytime(vopp_agent *agent, const vopp_plan_params *params, double budget_s,
                                     vopp_plan_result *out, int32_t *depth_reached);
/* tau(b, a, o): propagate every particle under `action` (Philox purpose 3, time step t of
 * the agent), reweight by Z(obs | s', a), resample systematically when ESS < N/2.  obs is a
 * host pointer: NAV2D float[2], GRID/TOY2/CROWD int32[1].  On VOPP_E_DEGENERATE (every particle
 * has zero likelihood) the belief is left unchanged.  ess_out / resampled_out may be NULL. */
VOPP_API int vopp_belief_update(vopp_agent *agent, int32_t action, const void *obs, double *ess_out,
                       int32_t *resampled_out);
/* tau(b, a, o) (Sec. III-B) for n agents of ctx at once: each agent is updated exactly as
 * vopp_belief_update would update it (subtree reuse included), the SIR updates of all of
 * them in one launch (one CTA per agent, the same arithmetic and reduction order, so the
 * particles, weights, ancestors, ESS and resampling decisions are bit-identical to n single
 * calls).  agents[i] (each at most once), actions[i] and obs[i] (a host pointer, as for
 * vopp_belief_update) describe update i; status_out[i] receives its status (VOPP_OK, or
 * VOPP_E_DEGENERATE with that agent's belief unchanged), ess_out[i] / resampled_out[i] (may
 * be NULL) its ESS (-1 for an adopted subtree) and resampling flag.  Returns VOPP_OK when
 * every update succeeded, else the first failing status; VOPP_E_INVALID (nothing updated)
 * for bad arguments, an agent of another context or an agent listed twice.  Serving loops
 * use it to update every agent whose plan just finished with one launch and one
 * synchronisation. */
VOPP_API int vopp_belief_update_batch(vopp_ctx *ctx, int32_t n, vopp_agent *const *agents,
                                      const int32_t *actions, const void *const *obs,
                                      double *ess_out, int32_t *resampled_out,
                                      int32_t *status_out);
/* Subtree reuse (enable = 1; 0 turns it off and releases what the agent keeps).  The
 * paper rebuilds its tree at every step (Alg. 1); with reuse on, an agent keeps what its
 * last plan expanded and builds on it:
 *   - vopp_agent_plan / vopp_submit_agent keep the plan's tree on the device (its own
 *     memory from the stream-ordered pool, outside any server's in-flight budget) until the
 *     agent's next plan or belief update;
 *   - vopp_belief_update(a, o) looks for a root branch (a, k) of the kept tree whose sampled
 *     observation equals o exactly (lowest k; discrete observations match, continuous ones
 *     practically never do).  If there is one, its branch weight is not zero (log omega >
 *     -inf) and the tree's level 1 is materialised (depth >= 3), that child's particle set
 *     and normalised log weights become the belief as the
 *     tree holds them (no propagation, no resampling; *ess_out = -1, *resampled_out = 0, the
 *     time step still advances) and its materialised subtree is kept; otherwise the SIR
 *     update runs and nothing is kept;
 *   - the agent's plans from an adopted belief continue that subtree, with the same width W
 *     and as long as the keys stay in range (key level + depth <= 255, node indices below
 *     2^64): they draw their random numbers as the nodes they are in the kept tree (the
 *     kept tree's seed, not params->seed), take the root as it stands (terminal particles
 *     keep their weight: they add no reward or value), and take the materialised levels the
 *     subtree already has instead of expanding them (VOPP_FLAG_REUSED, reused_levels): the
 *     plan's kernels read them where the subtree holds them, and copies into the plan's own
 *     tree run beside its first expansion.  A
 *     reused plan therefore equals the subtree below the adopted branches of one tree that
 *     is that much deeper, and every reused plan from the same belief is the same plan.
 * Anytime and episode-mode plans of the agent neither keep nor continue trees.
 * enable: 0 off; 1 on for models with discrete observations (GRID, TOY2, CROWD) and off for
 * NAV2D, whose continuous observations practically never equal a sampled one (its plans
 * would pay for kept trees that are never adopted); 2 on for every model (a caller that
 * feeds back the trees' own sampled observations).  Other values: VOPP_E_INVALID. */
VOPP_API int vopp_agent_set_reuse(vopp_agent *agent, int32_t enable);
/* After a belief update: the adopted branch a*W + k (or -1 when the SIR update ran), the
 * materialised levels of the kept subtree (root included, 0 if none) and the key level of
 * its root (the depth of the adopted node in the tree its keys belong to).  Any pointer may
 * be NULL. */
VOPP_API int vopp_agent_reuse_info(const vopp_agent *agent, int32_t *adopted_slot,
                                   int32_t *kept_levels, int32_t *key_level);
/* ---- closed loop (Alg. 1: plan, execute, perceive, update the belief) ---------------- */
/* The environment: a true state held on the device as a single particle, stepped by the
 * model's own transition and observation processes with random numbers of its own (Philox
 * key = seed; purpose 5 transition words 0,1 and purpose 6 observation words 0,1; node word
 * = the environment's step count t, starting at 0).  state: host NAV2D float[2] (x, y),
 * GRID/TOY2 int32[1], CROWD 15 words (one particle of the root layout); copied at
 * creation.  Paper: Alg. 1 "execute action, perceive
 * observation"; the paper's environments are simulators of the same models. */
typedef struct vopp_env vopp_env;
/* Create an environment of `model` at `state` (see above); destroy with vopp_env_destroy. */
VOPP_API int vopp_env_create(vopp_model *model, const void *state, uint64_t seed, vopp_env **out);
/* One step under `action`: obs receives the observation (host NAV2D float[2], GRID/TOY2/CROWD
 * int32[1]), reward and terminal (1 when the new state is terminal; terminal states are
 * absorbing with reward 0) may be NULL.  VOPP_E_INVALID for an action outside [0, A). */
VOPP_API int vopp_env_step(vopp_env *env, int32_t action, void *obs, float *reward, int32_t *terminal);
/* Copy the true state to the host (same layout as at creation). */
VOPP_API int vopp_env_get_state(vopp_env *env, void *state);
VOPP_API void vopp_env_destroy(vopp_env *env);

typedef struct {
  int32_t steps;             /* actions executed                                          */
  int32_t terminated;        /* 1: the true state reached a terminal state                */
  int32_t status;            /* VOPP_OK, or the error that ended the episode early        */
  int32_t min_depth;         /* smallest search depth reached by a plan (anytime budgets) */
  double total_reward;       /* sum_t r_t                                                 */
  double discounted_return;  /* sum_t gamma^t r_t                                         */
  uint64_t particle_steps;   /* planning particle-steps over the episode                  */
  double plan_seconds;       /* wall time spent planning                                  */
} vopp_episode_result;
/* Run one episode of at most max_steps: at step t plan from the agent's belief with
 * params (seed params->seed + t; one full-width plan of params->depth, or with anytime != 0
 * the anytime plan up to params->depth within budget_s), execute the chosen action in env,
 * stop if the true state is terminal, else update the belief with the observation
 * (vopp_belief_update).  actions / rewards: optional host arrays [max_steps].  An error of a
 * step (e.g. VOPP_E_DEGENERATE: the observation has zero likelihood under every particle)
 * ends the episode; it is returned and recorded in out->status with the steps done so far. */
VOPP_API int vopp_run_episode(vopp_agent *agent, vopp_env *env, const vopp_plan_params *params,
                              int32_t max_steps, int32_t anytime, double budget_s,
                              vopp_episode_result *out, int32_t *actions, float *rewards);

/* Copy the agent's particles (NAV2D x then y as float[2N]; GRID/TOY2 int32[N]; CROWD 15 rows
 * of N words) and
 * normalised log weights out; ancestors (int32[N], may be NULL) of the last update. */
VOPP_API int vopp_agent_get_particles(vopp_agent *agent, void *states, float *log_weights,
                             int32_t *ancestors, uint32_t ptr_flags);
VOPP_API int vopp_agent_num_particles(const vopp_agent *agent);
VOPP_API void vopp_agent_destroy(vopp_agent *agent);

/* Belief update without any memory allocation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory when they update a belief
 * (fixed memory plans of real-time loops, HBM held entirely by another allocator, or code
 * that cannot afford an allocation's implicit device synchronisation).  It runs the same
 * SIR kernel as vopp_belief_update, in place, on caller-owned device arrays:
 *   states       device, in/out: NAV2D float[2n] (x then y), GRID/TOY2 int32[n], CROWD
 *                15 rows of n words (robot x, y, 12 people coordinates, int32 flags)
 *   log_weights  device, in/out: normalised log weights float[n]
 *   obs          host: NAV2D float[2], GRID/TOY2/CROWD int32[1]
 *   seed, t      the Philox key and time step (counter) of this update
 *   cuda_stream  stream to run on (cudaStream_t as an integer, 0 = legacy default)
 *   ancestors    device int32[n] receiving the ancestor indices, or NULL
 *   ess_out, resampled_out   host, may be NULL
 * Its working memory is one static device array of about 1.5 MB compiled into the library
 * (every GPU that loads the library holds it until the process exits), so n is limited to
 * 65536 (CROWD, with 60-byte states: 20695); larger n returns VOPP_E_INVALID.  states,
 * log_weights and ancestors must be device memory of the model's GPU (checked with
 * cudaPointerGetAttributes; VOPP_E_INVALID otherwise); their sizes cannot be checked here,
 * so they must hold n particles as laid out above.  The call issues no cudaMalloc /
 * cudaFree and no allocating library call.  The first call on a device does a one-time
 * set-up: it looks the array's device address up (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share the one
 * array, which keeps the previous call's contents, so calls that overlap on the GPU
 * (different streams or threads, or concurrent launches) race: serialise them.  The call
 * reads the kernel's status word back and waits on cuda_stream, so it returns after the
 * update is done; the caller's current device is left as it was.  VOPP_E_DEGENERATE
 * leaves the belief unchanged. */
VOPP_API int vopp_belief_update_noalloc(const vopp_model *model, void *states, float *log_weights,
                                        int32_t n, int32_t action, const void *obs, uint64_t seed,
                                        uint64_t t, uintptr_t cuda_stream, int32_t *ancestors,
                                        double *ess_out, int32_t *resampled_out);

/* ---- batches: many uneven plans per launch sequence ----------------------------------- */
/* Run n independent plans with one launch per stage covering every plan (plans of
 * different models, N, D and W mix freely).  Results equal those of n separate vopp_plan
 * calls with the same arguments.  All models must belong to ctx. */
VOPP_API int vopp_plan_batch(vopp_ctx *ctx, int32_t n, const vopp_plan_request *reqs,
                    vopp_plan_result *outs);

/* ---- serving: continuous batching of plan requests ------------------------------------ */
typedef struct vopp_server vopp_server;
typedef struct {
  uint64_t submitted, completed, rejected;  /* rejected: footprint larger than the budget  */
  uint64_t batches, batched_plans, max_batch_seen;
  uint64_t particle_steps;                  /* of completed plans                         */
  uint64_t pending;                         /* requests waiting for a slot                */
  uint64_t in_flight_bytes, peak_in_flight_bytes;
} vopp_server_stats;

/* Start a serving loop on ctx: a worker thread batches queued requests (at most max_batch
 * per batch) onto n_slots streams whenever a slot is free and the batch's device footprint
 * fits in hbm_budget_bytes together with the batches already in flight (0 = the context's
 * budget); batches on different slots overlap on the device, and requests arriving while
 * others run join the next batch.  Arenas come from the context's stream-ordered memory
 * pool.  Slot 0's stream has the device's highest priority and takes small batches.  The
 * worker polls (yielding the CPU) while batches are in flight and for 2 ms after the last
 * one ends, then sleeps until the next request: under steady load it occupies one host
 * core, which keeps a request's start and completion free of thread wake-ups.  A plan's result does not depend on the batch it ran in.  The worker reads the
 * context's options and the models; do not destroy a model, agent or the context while
 * requests that use them are outstanding, and do not update an agent's belief while a
 * request on that agent is outstanding. */
VOPP_API int vopp_server_create(vopp_ctx *ctx, int32_t max_batch, int32_t n_slots,
                                size_t hbm_budget_bytes, vopp_server **out);
/* Stop accepting work, finish everything queued or in flight, release the server. */
VOPP_API void vopp_server_destroy(vopp_server *srv);
/* Queue one plan (non-blocking).  Host inputs are copied at submission; device inputs are
 * read when the request's batch runs and must stay valid until the ticket completes. */
VOPP_API int vopp_submit(vopp_server *srv, const vopp_plan_request *req, uint64_t *ticket);
/* Queue a plan from an agent's device-resident belief (non-blocking). */
VOPP_API int vopp_submit_agent(vopp_server *srv, vopp_agent *agent, const vopp_plan_params *params,
                               uint64_t *ticket);
/* VOPP_E_BUSY while the ticket's plan is queued or running; otherwise the plan's status,
 * with its result (and submission-to-completion latency in seconds) written and the ticket
 * released. */
VOPP_API int vopp_poll(vopp_server *srv, uint64_t ticket, vopp_plan_result *out, double *latency_s);
/* Like vopp_poll, blocking up to timeout_s seconds (VOPP_E_TIMEOUT if still not done). */
VOPP_API int vopp_wait(vopp_server *srv, uint64_t ticket, double timeout_s, vopp_plan_result *out,
                       double *latency_s);
/* Wait up to timeout_s seconds for the next plan to finish, in completion order; writes its
 * ticket (and result and latency) and releases it.  Returns the plan's status, or
 * VOPP_E_TIMEOUT when nothing finished in time.  A timeout of at most 5 ms is spent spinning
 * on the calling thread (no sleep: a completion is seen within about a microsecond, for a
 * serving loop that waits for its next completion or arrival); longer timeouts sleep. */
VOPP_API int vopp_wait_any(vopp_server *srv, double timeout_s, uint64_t *ticket,
                           vopp_plan_result *out, double *latency_s);
VOPP_API int vopp_server_get_stats(vopp_server *srv, vopp_server_stats *out);
/* paused = 1: keep queueing requests but start no new batch (batches in flight finish);
 * paused = 0: resume.  Lets a caller release a burst of requests as full batches. */
VOPP_API int vopp_server_set_paused(vopp_server *srv, int paused);

/* ---- autotuning ------------------------------------------------------------------------ */
typedef struct {
  int32_t leaf_threads;      /* chosen threads per leaf CTA (warps = branches processed at once) */
  int32_t persistent;        /* chosen leaf scheduling: 1 persistent CTAs, 0 one CTA per node   */
  double best_ms;            /* best time of the representative batch                         */
  int32_t n_tried;
  int32_t tried_threads[8], tried_persistent[8];
  double tried_ms[8];
} vopp_tune_result;
/* Time a representative batch (n requests, `reps` timed runs each) under every leaf
 * configuration -- 64 / 128 / 256 threads per leaf CTA, i.e. 2 / 4 / 8 branches per node in
 * flight, each with per-node or persistent scheduling -- check that all of them agree
 * within 1e-4 (they only reorder FP32 sums), and keep the fastest on the context. */
VOPP_API int vopp_autotune(vopp_ctx *ctx, int32_t n, const vopp_plan_request *reqs, int32_t reps,
                           vopp_tune_result *out);

/* ---- measurement aid (no counterpart in the paper) ----------------------------------- */
/* Issue rate of one arithmetic operation the leaf kernel is built from. */
typedef struct {
  char op[32];                          /* PTX operation measured, or "philox4x32-10 call"  */
  double thread_ops_per_clock_per_sm;   /* per SM cycle (clock64), independent of the clock */
  double ops_per_second;                /* whole device, at the clock of the moment         */
  int32_t sms;
} vopp_pipe_rate;
/* Microbenchmark: for each of up to max_out operations (FP32 FMA, packed f32x2 FMA, 32-bit
 * multiply-add (low and high half), three-input XOR, add, ex2, lg2, sin, sqrt, rsqrt, one
 * Philox4x32-10 call) run 4 CTAs x 256 threads per SM, 8 chains of 4096 steps
 * per thread, and report the rate.  Fills out[0 .. *n_out-1].  Allocates a few hundred KB
 * of device memory for the duration of the call and runs on its own stream; VOPP_E_CUDA
 * on a CUDA failure. */
VOPP_API int vopp_pipe_rates(int device, vopp_pipe_rate *out, int32_t max_out, int32_t *n_out);

/* The message of the last failing call on the calling thread (thread-local; valid until that
 * thread's next failing call). */
VOPP_API const char *vopp_last_error(void);
/* Library version string. */
VOPP_API const char *vopp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VOPP_H */
