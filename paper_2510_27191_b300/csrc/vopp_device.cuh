// vopp_device.cuh -- device-side building blocks of the VOPP hot path on sm_103a.
//
// Philox4x32-10 counter RNG, the uniform / Gaussian conventions, the three generative
// models (G(s,a) -> (s', o, r) of Sec. III-B, with their observation likelihoods and leaf
// heuristics), compensated sums and warp / block reductions, and the plan descriptor that
// the expansion and backup kernels read.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace vopp {

constexpr int kMaxDepth = 8;
constexpr int kMaxActions = 16;
constexpr int kMaxAW = 256;           // actions x branches per node
constexpr int kGridD2 = 256;          // squared agent-rock distances 0..221 (table padded)
constexpr int kNav = 0, kGrid = 1, kToy = 2, kCrowd = 3;
constexpr int kSample = 0, kEnumerate = 1;
constexpr int kPiUniform = 0, kPiFixed = 1, kPiNavDist = 2;

// Philox purposes (high byte of counter word 0).
constexpr uint32_t kPurposeTransition = 0, kPurposeObservation = 1, kPurposeBeliefStep = 3,
                   kPurposeResample = 4, kPurposeEnvStep = 5, kPurposeEnvObs = 6;

// Device status bits.
constexpr uint32_t kStatusDegenerateRoot = 1u;

// ---------------------------------------------------------------------------------------
// Constant tables of one model, built on the host at model creation.
// ---------------------------------------------------------------------------------------
struct DevModel {
  int kind, A, n_obs, branch_mode, pi_mode, h_zero;
  float pi_temp;
  float log_pi_fixed[kMaxActions];
  int rock_x[8], rock_y[8];
  int rock_at[121];                     // GRID: rock index of cell x + 11 y, or -1
  unsigned long long thr[kGridD2];      // GRID: floor(acc(d2) 2^32), acc(0) -> 2^32
  float lacc[kGridD2], l1macc[kGridD2]; // GRID: log acc, log(1 - acc)   (-inf at acc = 1)
  float lacc2[kGridD2], l1macc2[kGridD2]; // the same in base 2
  float pz[2 * kGridD2];                 // GRID: acc, then 1 - acc
  unsigned long long toy_thr;           // TOY2: floor(0.85 2^32)
  float toy_lc, toy_lw;                 // TOY2: log 0.85, log 0.15
  float toy_lc2, toy_lw2;               // TOY2: log2 0.85, log2 0.15
  float toy_pc, toy_pw;                 // TOY2: 0.85, 0.15
};

// The GRID expansion indexes log2 Z as lacc2[d^2 + 256 * disagree].
static_assert(offsetof(DevModel, l1macc2) == offsetof(DevModel, lacc2) + sizeof(float) * kGridD2,
              "l1macc2 follows lacc2");

struct DevResult {
  int status;                 // kStatus* bits
  int action;
  unsigned flags;
  unsigned degenerate;        // number of (node, action) pairs with vanished branch weights
  double v_root;
  double q[kMaxActions];
  double policy[kMaxActions];
};

// Everything one plan's kernels need.  Level l has nodes(l) = AW^l belief nodes; the
// child of node n through slot a*W + k is n*AW + a*W + k.
struct PlanDesc {
  int kind, A, W, AW, N, D, branch_mode, pi_mode, h_zero;
  int leaf_gen;               // 1: level D-1 particles are generated in the leaf kernel
  int keep_leaf;              // store branch stats at level D
  int keep_debug;             // store representatives / observations
  int fp64_root;              // back the root up in FP64 (else FP32, compensated)
  float eta, inv_eta, gamma, pi_temp;
  float log_pi[kMaxActions];  // uniform / fixed reference policy
  float h_a0, h_b0, log2_gamma;  // NAV2D / CROWD heuristic: h = a0 + b0 gamma^(m-1)
  uint32_t key0, key1;
  const DevModel *model;
  // root input (device copy or caller device pointer)
  const float *root_x, *root_y;
  const int *root_s;
  const float *root_w;        // linear weights (or null = uniform)
  const float *root_lw;       // log weights (agents); overrides root_w when set
  const float *root_pf;       // CROWD people [12][N] (rows 2q, 2q+1 = person q's x, y)
  // particle stores per level (levels 0 .. D-1, only those materialised)
  float *px[kMaxDepth], *py[kMaxDepth], *plw[kMaxDepth];
  int *ps[kMaxDepth];
  float *pf[kMaxDepth];       // CROWD people [node][12][N]
  // per-node / per-child arrays
  float *rbar[kMaxDepth + 1], *lom[kMaxDepth + 1], *V[kMaxDepth + 1];
  float *Q[kMaxDepth];
  float *mu[kMaxDepth];       // weighted mean particle (x,y) per node, kPiNavDist only
  int *rep[kMaxDepth + 1];
  float *obs[kMaxDepth + 1];  // 2 floats per child
  unsigned int *cnt[kMaxDepth];  // per node of levels 0..D-2: children finished (backup climb),
                                 // counted modulo A*W so that later iterations need no reset
  // anytime iterative deepening: preferences Psi [nodes][A] per internal level that persist
  // across iterations (null: one-pass closed form); levels >= psi_new_level are new
  float *psi[kMaxDepth];
  int psi_new_level;
  // Subtree reuse: a plan that continues a kept subtree keys its random numbers as the
  // nodes they are in the tree it continues (level l + lvl_off, index node + node_off[l],
  // node_off[l] = root index there x (A W)^l), and its root is that tree's node as it
  // stands (reuse_root: level 0 already holds its particles and normalised log weights).
  int lvl_off, reuse_root;
  unsigned long long node_off[kMaxDepth + 1];
  // the level-0 expansion prepares the root itself (no separate root preparation launch)
  int root_fused;
  // a plan continuing a kept subtree: its level-0 copies (entries copy0_first ..
  // copy0_first + copy0_n - 1 of the batch's copy table), made by its root preparation CTA
  int copy0_first, copy0_n;
  DevResult *result;
};

// Philox counter words of tree level l and node `node` of a plan (see PlanDesc).
__device__ __forceinline__ uint32_t key_level(const PlanDesc &P, int l) {
  return (uint32_t)(l + P.lvl_off);
}
__device__ __forceinline__ unsigned long long key_node(const PlanDesc &P, int l,
                                                       unsigned long long node) {
  return node + P.node_off[l];
}

// A launch covers work items of several plans: plan i owns items [prefix[i], prefix[i+1]).
struct StageTable {
  int n_plans;
  int level;                  // level of the work items (meaning depends on the kernel)
  const int *plan;            // [n_plans] plan index into the descriptor array
  const long long *prefix;    // [n_plans + 1]
  const int *levels;          // [n_plans] per-plan level (overrides `level` when non-null)
  unsigned long long *counter;  // persistent launches: next work item (zero at launch)
  // A copy tail: blocks >= work_grid of the launch copy 64 KB slices (copy_slices per entry)
  // of the n_copies entries of a CopyDesc table instead of taking work items (copies == null:
  // no tail, every block takes work items).
  const void *copies;
  int n_copies;
  unsigned copy_slices;
  unsigned work_grid;
};

__device__ __forceinline__ int find_plan(const StageTable &st, long long item) {
  int lo = 0, hi = st.n_plans - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (st.prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter words:
//   c0 = level | action << 8 | branch << 16, c1 = idx | purpose << 24, (c2, c3) = node.
// The word that varies across a loop's particles (idx) is c1, which the first round does not
// multiply: with the other words fixed in a loop, the first two rounds' products of c0 and
// c2 are loop-invariant (two wide multiplies fewer per call).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // each round's two 32x32 -> 64-bit products as single wide multiplies
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                   (uint32_t)p0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the round keys (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85) taken from a
// table (rk[r] = round r's key pair), e.g. one a CTA fills once in shared memory.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint2 *rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint2 k = rk[r];
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y,
                   (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint32_t idx, uint32_t purpose,
                                      uint32_t level, uint32_t a, uint32_t k,
                                      unsigned long long node) {
  return philox(make_uint4(level | (a << 8) | (k << 16), idx | (purpose << 24),
                           (uint32_t)node, (uint32_t)(node >> 32)),
                k0, k1);
}

// Two-wide FP32 arithmetic (Blackwell packed f32x2 FMA / ADD / MUL on float2), used to run
// the two particles of a Philox pair through the same instruction.
#ifndef VOPP_SCALAR2
#define VOPP_SCALAR2 0
#endif
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
#if VOPP_SCALAR2
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y)); }
#else
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
#endif

// u = (2 (x >> 9) + 1) 2^-24: exact in FP32, strictly inside (0, 1).  Built from the float
// 1 + (x >> 9) 2^-23 in [1, 2) minus (1 - 2^-24); the difference is representable, so the
// subtraction is exact.
// The bits of 1 + (x >> 9) 2^-23.
__device__ __forceinline__ uint32_t u01_bits(uint32_t x) { return (x >> 9) | 0x3F800000u; }
__device__ __forceinline__ float u01(uint32_t x) {
  return __fadd_rn(__uint_as_float(u01_bits(x)), -0.999999940395355225f);
}
__device__ __forceinline__ float2 u01_2(uint32_t a, uint32_t b) {
  return add2(make_float2(__uint_as_float(u01_bits(a)), __uint_as_float(u01_bits(b))),
              bc2(-0.999999940395355225f));
}

// Hardware base-2 exponential / logarithm (PTX ex2.approx / lg2.approx, flush-to-zero):
// ex2(-inf) = +0, lg2(+0) = -inf.
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Hardware reciprocal (PTX rcp.approx, flush-to-zero).
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Hardware square root (PTX sqrt.approx, flush-to-zero): one SFU operation where
// x * rsqrt(x) takes an SFU operation and a multiply.
__device__ __forceinline__ float sqrta(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1.0f if a <= b, else 0.0f (PTX set with a float destination: one compare, no select).
__device__ __forceinline__ float setle1(float a, float b) {
  float y;
  asm("set.le.f32.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
  return y;
}

// fma(a, b, c) saturated to [0, 1] (PTX fma.rn.sat: an FMA-pipe instruction).
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
  float y;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
  return y;
}
#ifndef VOPP_NAV_CLAMP_SAT
#define VOPP_NAV_CLAMP_SAT 1
#endif
#ifndef VOPP_NAV_ABS_FFMA
#define VOPP_NAV_ABS_FFMA 0
#endif
#ifndef VOPP_NAV_HEUR_SAT
#define VOPP_NAV_HEUR_SAT 0
#endif

// max(a, b, c) in one instruction (three-input max of sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float y;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
  return y;
}
constexpr float kLog2e = 1.44269504088896341f;
constexpr float kLn2 = 0.693147180559945309f;


// -2 ln(u) for u in (0, 1).  Where -ln u > 2^-8 the hardware base-2 logarithm (absolute
// error ~2^-22) gives a relative error below 5e-5 that shrinks as u moves away from 1;
// for u > 1 - 2^-8 the Taylor series -2 ln(1 - v) = 2 (v + v^2/2 + v^3/3 + v^4/4)
// (v = 1 - u, exact) truncates below v^4 / 5 < 1e-10 relative.
__device__ __forceinline__ float neg2_log_u(float u) {
  const float v = fmaf(u, -1.0f, 1.0f);
  float ser = fmaf(v, 0.5f, 0.666666687f);
  ser = fmaf(v, ser, 1.0f);
  ser = fmaf(v, ser, 2.0f);
  ser = __fmul_rn(ser, v);
  const float hw = __fmul_rn(-1.38629436f, lg2(u));
  return (v < 0.00390625f) ? ser : hw;
}
// Two at once; the series is evaluated only when one of the two needs it (about one pair in
// 128), so the common case is the hardware logarithm and a product.
__device__ __forceinline__ float2 neg2_log_u2(float2 u) {
  float2 r = mul2(bc2(-1.38629436f), make_float2(lg2(u.x), lg2(u.y)));
  const bool nx = u.x > 0.99609375f, ny = u.y > 0.99609375f;   // v = 1 - u < 2^-8
  if (nx || ny) {
    const float2 v = fma2(u, bc2(-1.0f), bc2(1.0f));
    float2 ser = fma2(v, bc2(0.5f), bc2(0.666666687f));
    ser = fma2(v, ser, bc2(1.0f));
    ser = fma2(v, ser, bc2(2.0f));
    ser = mul2(ser, v);
    r = make_float2(nx ? ser.x : r.x, ny ? ser.y : r.y);
  }
  return r;
}

// Box-Muller: (g1, g2) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).  The angle is taken as
// t = 2 pi u2 - pi in (-pi, pi), where the hardware sine / cosine are accurate, and
// cos(2 pi u2) = -cos t, sin(2 pi u2) = -sin t; the returned pair is (-g1, -g2)'s negation
// folded in: the caller gets r cos t and r sin t and subtracts.
__device__ __forceinline__ float2 box_muller_neg(uint32_t a, uint32_t b) {
  const float u1 = u01(a), u2 = u01(b);
  const float s = neg2_log_u(u1);
  const float r = sqrta(s);
  const float t = fmaf(6.28318531f, u2, -3.14159265f);
  float sn, cs;
  __sincosf(t, &sn, &cs);
  return make_float2(__fmul_rn(r, cs), __fmul_rn(r, sn));   // = (-g1, -g2)
}
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
  const float2 n = box_muller_neg(a, b);
  return make_float2(-n.x, -n.y);
}

// ---------------------------------------------------------------------------------------
// Compensated (Kahan) accumulation and online log-sum-exp.
// ---------------------------------------------------------------------------------------
struct Kahan {
  float s, c;
  __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ void scale(float f) { s *= f; c *= f; }
  __device__ __forceinline__ float value() const { return __fsub_rn(s, c); }
};

// Streaming sum of exp(L_i - m) (and of exp(L_i - m) h_i) with a running maximum m.
struct OnlineLSE {
  float m;
  Kahan s, h;
  __device__ __forceinline__ void init() { m = -CUDART_INF_F; s.init(); h.init(); }
  __device__ __forceinline__ void add(float L, float hv) {
    if (!(L > -CUDART_INF_F)) return;            // zero weight contributes nothing
    if (L > m) {
      const float t = __expf(m - L);             // 0 when m = -inf
      s.scale(t); h.scale(t);
      m = L;
      s.add(1.0f); h.add(hv);
    } else {
      const float t = __expf(L - m);
      s.add(t); h.add(t * hv);
    }
  }
  __device__ __forceinline__ void add(float L) {
    if (!(L > -CUDART_INF_F)) return;
    if (L > m) {
      const float t = __expf(m - L);
      s.scale(t);
      m = L;
      s.add(1.0f);
    } else {
      s.add(__expf(L - m));
    }
  }
};

// Warp-wide merge of per-lane max-shifted sums (m, s, h): the lanes agree on the largest
// shift M first, rescale by 2^(m - M) (base-2 shifts) and add.  Every lane gets the result.
__device__ __forceinline__ void warp_lse2(float &m, float &s, float &h) {
  float M = m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
  const float f = (m > -CUDART_INF_F) ? ex2(m - M) : 0.f;
  s *= f;
  h *= f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    h += __shfl_xor_sync(0xffffffffu, h, o);
  }
  m = M;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Four warp sums at once: the halves of the warp exchange two values, the quarters one, so
// that 10 shuffles (5 exchanges, 4 broadcasts) replace 20; every lane gets the four totals.
__device__ __forceinline__ void warp_sum4(float a, float b, float c, float d, float &sa,
                                          float &sb, float &sc, float &sd) {
  const unsigned F = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool hi = (lane & 16) != 0, h8 = (lane & 8) != 0;
  float k0 = hi ? c : a, k1 = hi ? d : b;                 // kept: (a, b) low half, (c, d) high
  k0 += __shfl_xor_sync(F, hi ? a : c, 16);
  k1 += __shfl_xor_sync(F, hi ? b : d, 16);
  float k = h8 ? k1 : k0;                                  // lanes 0-7 a, 8-15 b, 16-23 c, 24-31 d
  k += __shfl_xor_sync(F, h8 ? k0 : k1, 8);
  k += __shfl_xor_sync(F, k, 4);
  k += __shfl_xor_sync(F, k, 2);
  k += __shfl_xor_sync(F, k, 1);
  sa = __shfl_sync(F, k, 0);
  sb = __shfl_sync(F, k, 8);
  sc = __shfl_sync(F, k, 16);
  sd = __shfl_sync(F, k, 24);
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reductions (every thread gets the result).  `red` holds >= 32 floats.
__device__ __forceinline__ float block_sum(float v, float *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = (lane < nw) ? red[lane] : 0.f;
  t = warp_sum(t);
  return t;
}

// Four block-wide sums at once (every thread gets them).  `red` holds >= 128 floats.
__device__ __forceinline__ void block_sum4(float (&v)[4], float *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) red[32 * k + wid] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = warp_sum((lane < nw) ? red[32 * k + lane] : 0.f);
}

__device__ __forceinline__ float block_max(float v, float *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = (lane < nw) ? red[lane] : -CUDART_INF_F;
  return warp_max(t);
}

// ---------------------------------------------------------------------------------------
// Models.  Each provides: a particle type, step (transition + reward, absorbing terminals),
// draw_obs (o ~ Z(.|s',a) from Philox words), loglik (log Z(o|s',a), -inf if impossible)
// and heuristic (leaf ValueHeuristic of Alg. 2).
// ---------------------------------------------------------------------------------------
struct NavModel {
  static constexpr bool kStochastic = true;
  static constexpr bool kPairPacked = true;
  struct S { float x, y; };
  struct O { float x, y; };

  __device__ __forceinline__ static bool terminal(const S &s) {
    return fmaf(s.x, s.x, __fmul_rn(s.y, s.y)) <= 0.25f;
  }
  __device__ __forceinline__ static float dx_of(int a) { return (a == 0) ? 1.0f : ((a == 1) ? -1.0f : 0.0f); }
  __device__ __forceinline__ static float dy_of(int a) { return (a == 2) ? 1.0f : ((a == 3) ? -1.0f : 0.0f); }
  // Transition s' = clamp(s + delta_a + 0.1 g, 0, 10); reward +100 on entering the goal disc,
  // -1 otherwise; terminal states stay put with reward 0.
  __device__ __forceinline__ static float step(S &s, int a, uint32_t wa, uint32_t wb,
                                               const DevModel &) {
    const bool term = fmaf(s.x, s.x, __fmul_rn(s.y, s.y)) <= 0.25f;
    const float2 ng = box_muller_neg(wa, wb);
    const float nx = fminf(fmaxf(fmaf(-0.1f, ng.x, __fadd_rn(s.x, dx_of(a))), 0.0f), 10.0f);
    const float ny = fminf(fmaxf(fmaf(-0.1f, ng.y, __fadd_rn(s.y, dy_of(a))), 0.0f), 10.0f);
    const float r = (fmaf(nx, nx, __fmul_rn(ny, ny)) <= 0.25f) ? 100.0f : -1.0f;
    s.x = term ? s.x : nx;
    s.y = term ? s.y : ny;
    return term ? 0.0f : r;
  }
  // The two particles of a Philox pair (x = (x0, x1), y = (y0, y1), words w) stepped with
  // two-wide arithmetic; same operation sequence as step().  Returns the rewards; terminal
  // flags of the new states in t0 / t1.
  __device__ __forceinline__ static float2 step_pair(float2 &x, float2 &y, float dx, float dy,
                                                     uint4 w, bool &t0, bool &t1) {
    const float2 rr = fma2(x, x, mul2(y, y));
    const bool p0 = rr.x <= 0.25f, p1 = rr.y <= 0.25f;
    const float2 u1 = u01_2(w.x, w.z), u2 = u01_2(w.y, w.w);
    const float2 sq = neg2_log_u2(u1);
    const float2 r = make_float2(sqrta(sq.x), sqrta(sq.y));
    const float2 t = fma2(bc2(6.28318531f), u2, bc2(-3.14159265f));
    float s0, c0, s1, c1;
    __sincosf(t.x, &s0, &c0);
    __sincosf(t.y, &s1, &c1);
#if VOPP_NAV_CLAMP_SAT
    // The same values with the lower clamp on the FMA pipe: in units of 16 (a power of two,
    // so every scaling is exact) the step is t = fma(-0.1 / 16, r cos, (x + dx) / 16) =
    // nx / 16 exactly, a saturating FMA gives max(t, 0) (t < 1: |nx| < 16), and 16 max(t, 0)
    // = max(nx, 0); only the upper clamp stays a min on the half-rate ALU pipe.
    const float2 wx = fma2(x, bc2(0.0625f), bc2(0.0625f * dx));
    const float2 wy = fma2(y, bc2(0.0625f), bc2(0.0625f * dy));
    const float2 rc = mul2(r, make_float2(c0, c1)), rs = mul2(r, make_float2(s0, s1));
    float2 nx = mul2(bc2(16.0f), make_float2(fma_sat(rc.x, -0.00625f, wx.x),
                                             fma_sat(rc.y, -0.00625f, wx.y)));
    float2 ny = mul2(bc2(16.0f), make_float2(fma_sat(rs.x, -0.00625f, wy.x),
                                             fma_sat(rs.y, -0.00625f, wy.y)));
    nx = make_float2(fminf(nx.x, 10.0f), fminf(nx.y, 10.0f));
    ny = make_float2(fminf(ny.x, 10.0f), fminf(ny.y, 10.0f));
#else
    float2 nx = fma2(bc2(-0.1f), mul2(r, make_float2(c0, c1)), add2(x, bc2(dx)));
    float2 ny = fma2(bc2(-0.1f), mul2(r, make_float2(s0, s1)), add2(y, bc2(dy)));
    nx = make_float2(fminf(fmaxf(nx.x, 0.0f), 10.0f), fminf(fmaxf(nx.y, 0.0f), 10.0f));
    ny = make_float2(fminf(fmaxf(ny.x, 0.0f), 10.0f), fminf(fmaxf(ny.y, 0.0f), 10.0f));
#endif
    const float2 r2 = fma2(nx, nx, mul2(ny, ny));
    const bool g0 = r2.x <= 0.25f, g1 = r2.y <= 0.25f;
    x = make_float2(p0 ? x.x : nx.x, p1 ? x.y : nx.y);
    y = make_float2(p0 ? y.x : ny.x, p1 ? y.y : ny.y);
    t0 = p0 || g0;
    t1 = p1 || g1;
    return make_float2(p0 ? 0.0f : (g0 ? 100.0f : -1.0f), p1 ? 0.0f : (g1 ? 100.0f : -1.0f));
  }
  // The leaf's pair step on positions in units of 16 (x / 16, y / 16: power-of-two scalings,
  // so every value below is 1/16 of step_pair's, bit for bit, and the clamp's upper bound is
  // 10 / 16).  m = (m0, m1): 1 for a live particle, 0 for a terminal one, which then draws
  // no noise and takes no move (x + m dx + m r cos = x), and earns m (101 gm - 1) = 0.
  // gm: 1.0 where the new state is in the goal disc (x^2 + y^2 <= 1/4, i.e. 2^-10 in these
  // units), else 0.0 -- also 1 for every terminal particle, which sits in the disc.  No
  // selects: the masks enter as FMA operands.  Returns the rewards.
  __device__ __forceinline__ static float2 step_pair16(float2 &x, float2 &y, float dx16,
                                                       float dy16, uint4 w, float2 m,
                                                       float2 &gm) {
    const float2 u1 = u01_2(w.x, w.z), u2 = u01_2(w.y, w.w);
    const float2 sq = mul2(neg2_log_u2(u1), m);
    const float2 r = make_float2(sqrta(sq.x), sqrta(sq.y));
    const float2 t = fma2(bc2(6.28318531f), u2, bc2(-3.14159265f));
    float s0, c0, s1, c1;
    __sincosf(t.x, &s0, &c0);
    __sincosf(t.y, &s1, &c1);
    const float2 wx = fma2(m, bc2(dx16), x), wy = fma2(m, bc2(dy16), y);
    const float2 rc = mul2(r, make_float2(c0, c1)), rs = mul2(r, make_float2(s0, s1));
    // the lower clamp as a saturating FMA (values below 1 here), the upper one a min
    float2 nx = make_float2(fma_sat(rc.x, -0.00625f, wx.x), fma_sat(rc.y, -0.00625f, wx.y));
    float2 ny = make_float2(fma_sat(rs.x, -0.00625f, wy.x), fma_sat(rs.y, -0.00625f, wy.y));
    nx = make_float2(fminf(nx.x, 0.625f), fminf(nx.y, 0.625f));
    ny = make_float2(fminf(ny.x, 0.625f), fminf(ny.y, 0.625f));
    const float2 r2 = fma2(nx, nx, mul2(ny, ny));
    gm = make_float2(setle1(r2.x, 0.0009765625f), setle1(r2.y, 0.0009765625f));
    x = nx;
    y = ny;
    return mul2(fma2(gm, bc2(101.0f), bc2(-1.0f)), m);
  }
  // zlin_pair on positions in units of 16 (x - 9 = fma(x16, 16, -9) and o - x =
  // fma(x16, -16, o) round exactly as the unscaled forms).
  __device__ __forceinline__ static float2 zlin_pair16(float2 x, float2 y, const O &o) {
    const float2 dm = fma2(x, bc2(16.0f), bc2(-9.0f));
    const float2 sc = fma2(bc2(0.588705011f), make_float2(fabsf(dm.x), fabsf(dm.y)),
                           bc2(0.0588705011f));          // (0.5 |x - 9| + 0.05) / sqrt(c)
    const float2 s2 = mul2(sc, sc);
    const float2 pk = make_float2(rcpa(s2.x), rcpa(s2.y));
    const float2 ex = fma2(x, bc2(-16.0f), bc2(o.x)), ey = fma2(y, bc2(-16.0f), bc2(o.y));
    const float2 d2 = fma2(ex, ex, mul2(ey, ey));
    const float2 q = mul2(d2, make_float2(-pk.x, -pk.y));
    return mul2(make_float2(ex2(q.x), ex2(q.y)), pk);
  }
  // heuristic_pair on positions in units of 16; zero where gm = 1 (goal reached or terminal:
  // h - h gm), and everywhere when a0 = b0 = 0 (the forced-zero heuristic).
  __device__ __forceinline__ static float2 heuristic_pair16(float2 x, float2 y, float2 gm,
                                                            float log2g, float a0, float b0) {
    float2 v = add2(x, y);                                // (x + y) / 16
    v = make_float2(fmaxf(v.x, 0.09375f), fmaxf(v.y, 0.09375f));
    const float2 e = fma2(v, bc2(16.0f * log2g), bc2(-1.5f * log2g));
    const float2 h = fma2(bc2(b0), make_float2(ex2(e.x), ex2(e.y)), bc2(a0));
    return fma2(make_float2(-h.x, -h.y), gm, h);
  }
  __device__ __forceinline__ static float sigma(float x) {
    return fmaf(0.5f, fabsf(__fadd_rn(x, -9.0f)), 0.05f);
  }
  __device__ __forceinline__ static O draw_obs(const S &s, int, uint32_t w0, uint32_t w1,
                                               const DevModel &) {
    const float2 g = box_muller(w0, w1);
    const float sg = sigma(s.x);
    return O{fmaf(sg, g.x, s.x), fmaf(sg, g.y, s.y)};
  }
  // Base-2 log-likelihoods of observation o for the two particles of a pair.
  // 1/sigma^2 comes from the same logarithm, 2^(-2 log2 sigma): one ex2 instead of a
  // reciprocal and a product.
  __device__ __forceinline__ static float2 loglik2_pair(float2 x, float2 y, const O &o) {
    const float2 dm = add2(x, bc2(-9.0f));
    const float2 sg = fma2(bc2(0.5f), make_float2(fabsf(dm.x), fabsf(dm.y)), bc2(0.05f));
    const float2 lg = make_float2(lg2(sg.x), lg2(sg.y));
    // -2 log2 sigma - log2(2 pi), and log2(log2(e) / 2) - 2 log2 sigma whose 2^ is
    // log2(e) / (2 sigma^2), the factor of -|o - s'|^2
    const float2 t = fma2(lg, bc2(-2.0f), bc2(-2.65149613f));
    const float2 f = fma2(lg, bc2(-2.0f), bc2(-0.471233627f));
    const float2 is2 = make_float2(-ex2(f.x), -ex2(f.y));
    const float2 ex = fma2(x, bc2(-1.0f), bc2(o.x)), ey = fma2(y, bc2(-1.0f), bc2(o.y));
    const float2 d2 = fma2(ex, ex, mul2(ey, ey));
    return fma2(d2, is2, t);
  }
  // The likelihoods of observation o for the two particles of a pair in linear form, up to
  // one factor common to all particles: with c = log2(e) / 2 and pk = c / sigma^2,
  // Z(o | s') = 2^(-|o - s'|^2 pk) pk / (2 pi c).  The factor 1 / (2 pi c) is dropped.
  // sigma / sqrt(c) comes from one fused multiply-add, pk from one reciprocal.
  __device__ __forceinline__ static float2 zlin_pair(float2 x, float2 y, const O &o) {
    const float2 dm = add2(x, bc2(-9.0f));
#if VOPP_NAV_ABS_FFMA
    // scalar FMAs take |dm| as an operand modifier (no separate absolute value)
    const float2 sc = make_float2(fmaf(0.588705011f, fabsf(dm.x), 0.0588705011f),
                                  fmaf(0.588705011f, fabsf(dm.y), 0.0588705011f));
#else
    const float2 sc = fma2(bc2(0.588705011f), make_float2(fabsf(dm.x), fabsf(dm.y)),
                           bc2(0.0588705011f));          // (0.5 |x - 9| + 0.05) / sqrt(c)
#endif
    const float2 s2 = mul2(sc, sc);
    const float2 pk = make_float2(rcpa(s2.x), rcpa(s2.y));
    const float2 ex = fma2(x, bc2(-1.0f), bc2(o.x)), ey = fma2(y, bc2(-1.0f), bc2(o.y));
    const float2 d2 = fma2(ex, ex, mul2(ey, ey));
    const float2 q = mul2(d2, make_float2(-pk.x, -pk.y));
    return mul2(make_float2(ex2(q.x), ex2(q.y)), pk);
  }
  // Heuristic of the pair; t0 / t1 are the terminal flags of the states.
  __device__ __forceinline__ static float2 heuristic_pair(float2 x, float2 y, bool t0, bool t1,
                                                          float log2g, float a0, float b0, bool hz) {
    // m - 1 = max(x + y - 1/2, 1) - 1 = max(x + y, 3/2) - 3/2
#if VOPP_NAV_HEUR_SAT
    // max(v - 3/2, 0) = 20 sat((v - 3/2) / 20) for v = x + y <= 20: one saturating FMA
    const float2 v = add2(x, y);
    const float2 q = make_float2(fma_sat(v.x, 0.05f, -0.075f), fma_sat(v.y, 0.05f, -0.075f));
    const float2 e = mul2(q, bc2(20.0f * log2g));
#else
    float2 m = add2(x, y);
    m = make_float2(fmaxf(m.x, 1.5f), fmaxf(m.y, 1.5f));
    const float2 e = fma2(m, bc2(log2g), bc2(-1.5f * log2g));
#endif
    const float2 h = fma2(bc2(b0), make_float2(ex2(e.x), ex2(e.y)), bc2(a0));
    return make_float2((hz || t0) ? 0.0f : h.x, (hz || t1) ? 0.0f : h.y);
  }
  __device__ __forceinline__ static O enum_obs(int k) { return O{(float)k, 0.f}; }
  // log2 N(o; s', sigma(x')^2 I) = log2 e (-|o - s'|^2 / (2 sigma^2)) - 2 log2 sigma
  //                                 - log2(2 pi)
  __device__ __forceinline__ static float loglik2(const S &s, int, const O &o, const DevModel &) {
    const float sg = sigma(s.x);
    const float t = __fmul_rn(-2.0f, lg2(sg));      // -2 log2 sigma
    const float is2 = ex2(t);                       // 1 / sigma^2
    const float ex = fmaf(s.x, -1.0f, o.x), ey = fmaf(s.y, -1.0f, o.y);
    const float d2 = fmaf(ex, ex, __fmul_rn(ey, ey));
    return fmaf(__fmul_rn(-0.721347520f, d2), is2, __fadd_rn(t, -2.65149613f));
  }
  __device__ __forceinline__ static float loglik(const S &s, int a, const O &o, const DevModel &m) {
    return kLn2 * loglik2(s, a, o, m);
  }
  // h = a0 + b0 gamma^(m-1), m = max(1, x + y - 1/2); 0 at terminal states.  hz is 0 when
  // the heuristic is forced to zero, 1 otherwise.
  __device__ __forceinline__ static float heuristic(const S &s, float log2g, float a0, float b0,
                                                    bool hz) {
    const float m = fmaxf(__fadd_rn(__fadd_rn(s.x, s.y), -0.5f), 1.0f);
    const float h = fmaf(b0, ex2(fmaf(m, log2g, -log2g)), a0);
    return (hz || terminal(s)) ? 0.0f : h;
  }
  __device__ __forceinline__ static float heuristic(const S &s, const PlanDesc &P) {
    return heuristic(s, P.log2_gamma, P.h_a0, P.h_b0, P.h_zero != 0);
  }
  __device__ __forceinline__ static float2 obs_f2(const O &o) { return make_float2(o.x, o.y); }
};

__device__ __forceinline__ int gx(int s) { return (s >> 8) & 0xF; }
__device__ __forceinline__ int gy(int s) { return (s >> 12) & 0xF; }
__device__ __forceinline__ int gterm(int s) { return (s >> 16) & 1; }
__device__ __forceinline__ int gpack(int rocks, int x, int y, int t) {
  return (rocks & 0xFF) | (x << 8) | (y << 12) | (t << 16);
}

struct GridModel {
  static constexpr bool kStochastic = false;
  static constexpr bool kPairPacked = false;
  struct S { int s; };
  struct O { int o; };

  __device__ __forceinline__ static bool terminal(const S &s) { return gterm(s.s) != 0; }
  // The branch on the action is the same for a whole leaf branch; inside each action the
  // per-particle cases (terminal, exit, rock) are selects, not branches.  A non-terminal
  // state has bit 16 clear and x <= 10, so a move changes one field by one without a carry
  // (the exit sets x = 11 and the terminal bit together).
  __device__ __forceinline__ static float step(S &st, int a, uint32_t, uint32_t,
                                               const DevModel &m) {
    const int s = st.s;
    const bool term = gterm(s) != 0;
    const int x = gx(s), y = gy(s);
    int ns = s;
    float r = 0.0f;
    if (a == 0) {
      const bool exit_e = x == 10;
      ns = s + (exit_e ? 0x10100 : 0x100);
      r = exit_e ? 10.0f : 0.0f;
    } else if (a == 1) {
      ns = (x > 0) ? s - 0x100 : s;
    } else if (a == 2) {
      ns = (y < 10) ? s + 0x1000 : s;
    } else if (a == 3) {
      ns = (y > 0) ? s - 0x1000 : s;
    } else if (a == 4) {
      const int rk = (!term && x <= 10) ? m.rock_at[x + 11 * y] : -1;
      const bool on = rk >= 0, good = on && ((s >> (rk & 7)) & 1);
      r = on ? (good ? 10.0f : -10.0f) : 0.0f;
      ns = good ? (s & ~(1 << (rk & 7))) : s;
    }
    st.s = term ? s : ns;
    return term ? 0.0f : r;
  }
  __device__ __forceinline__ static int d2(const S &s, int rk, const DevModel &m) {
    const int dx = gx(s.s) - m.rock_x[rk], dy = gy(s.s) - m.rock_y[rk];
    return dx * dx + dy * dy;
  }
  __device__ __forceinline__ static O draw_obs(const S &s, int a, uint32_t w0, uint32_t,
                                               const DevModel &m) {
    if (a < 5) return O{0};
    const int rk = a - 5, bit = (s.s >> rk) & 1;
    const bool correct = (unsigned long long)w0 < m.thr[d2(s, rk, m)];
    const int seen = correct ? bit : 1 - bit;
    return O{seen ? 1 : 2};
  }
  __device__ __forceinline__ static O enum_obs(int k) { return O{k}; }
  __device__ __forceinline__ static float loglik(const S &s, int a, const O &o, const DevModel &m) {
    if (a < 5) return (o.o == 0) ? 0.0f : -CUDART_INF_F;
    if (o.o != 1 && o.o != 2) return -CUDART_INF_F;
    const int rk = a - 5, bit = (s.s >> rk) & 1;
    const int dd = d2(s, rk, m);
    return ((o.o == 1) == (bit == 1)) ? m.lacc[dd] : m.l1macc[dd];
  }
  __device__ __forceinline__ static float loglik2(const S &s, int a, const O &o, const DevModel &m) {
    if (a < 5) return (o.o == 0) ? 0.0f : -CUDART_INF_F;
    if (o.o != 1 && o.o != 2) return -CUDART_INF_F;
    const int rk = a - 5, bit = (s.s >> rk) & 1;
    const int dd = d2(s, rk, m);
    return ((o.o == 1) == (bit == 1)) ? m.lacc2[dd] : m.l1macc2[dd];
  }
  // Z(o | s') itself: one load from the [agree, disagree][d^2] table
  __device__ __forceinline__ static float zlin(const S &s, int a, const O &o, const DevModel &m) {
    if (a < 5) return (o.o == 0) ? 1.0f : 0.0f;
    if (o.o != 1 && o.o != 2) return 0.0f;
    const int rk = a - 5;
    const int miss = ((s.s >> rk) & 1) ^ (o.o == 1 ? 1 : 0);   // reading != the rock's bit
    return m.pz[miss * kGridD2 + d2(s, rk, m)];
  }
  __device__ __forceinline__ static float heuristic(const S &s, float log2g, float, float, bool hz) {
    const float h = 10.0f * ex2((float)(10 - gx(s.s)) * log2g);
    return (hz || gterm(s.s)) ? 0.0f : h;
  }
  __device__ __forceinline__ static float heuristic(const S &s, const PlanDesc &P) {
    return heuristic(s, P.log2_gamma, P.h_a0, P.h_b0, P.h_zero != 0);
  }
  __device__ __forceinline__ static float2 obs_f2(const O &o) { return make_float2((float)o.o, 0.f); }
};

struct ToyModel {
  static constexpr bool kStochastic = false;
  static constexpr bool kPairPacked = false;
  struct S { int s; };

  struct O { int o; };

  __device__ __forceinline__ static bool terminal(const S &) { return false; }
  __device__ __forceinline__ static float step(S &st, int a, uint32_t, uint32_t, const DevModel &) {
    const int s = st.s;
    st.s = (a == 1) ? 1 - s : s;
    return (a == 1) ? -0.1f : (s == 0 ? 1.0f : -1.0f);
  }
  __device__ __forceinline__ static O draw_obs(const S &s, int, uint32_t w0, uint32_t,
                                               const DevModel &m) {
    const bool correct = (unsigned long long)w0 < m.toy_thr;
    return O{correct ? s.s : 1 - s.s};
  }
  __device__ __forceinline__ static O enum_obs(int k) { return O{k}; }
  __device__ __forceinline__ static float loglik(const S &s, int, const O &o, const DevModel &m) {
    if (o.o != 0 && o.o != 1) return -CUDART_INF_F;
    return (o.o == s.s) ? m.toy_lc : m.toy_lw;
  }
  __device__ __forceinline__ static float loglik2(const S &s, int, const O &o, const DevModel &m) {
    if (o.o != 0 && o.o != 1) return -CUDART_INF_F;
    return (o.o == s.s) ? m.toy_lc2 : m.toy_lw2;
  }
  __device__ __forceinline__ static float zlin(const S &s, int, const O &o, const DevModel &m) {
    if (o.o != 0 && o.o != 1) return 0.0f;
    return (o.o == s.s) ? m.toy_pc : m.toy_pw;
  }
  __device__ __forceinline__ static float heuristic(const S &, float, float, float, bool) { return 0.0f; }
  __device__ __forceinline__ static float heuristic(const S &, const PlanDesc &) { return 0.0f; }
  __device__ __forceinline__ static float2 obs_f2(const O &o) { return make_float2((float)o.o, 0.f); }
};

// ---------------------------------------------------------------------------------------
// CROWD: the paper's CrowdNav problem (Sec. IV) as a synthetic model.  A robot in a 50 x 40 m
// hall and the six nearest people, each curious or shy (hidden).  Actions 0 NORTH, 1 EAST,
// 2 SOUTH, 3 WEST (1 m; the east, west and south walls hold the robot), 4 YELL.  Every person
// moves by N(0, 0.05^2) noise per axis; a person within 4 m of the robot's new position
// reacts with probability 0.9 -- curious 0.3 m toward it (never past it), shy 0.8 m away --
// and under YELL every such person backs away 2 m instead.  Reward -1 per step, -25 for
// YELL, -200 per person within 0.5 m after the step, +1000 on leaving north (terminal).
// Observation: per person whether it came closer to the robot's new position, read from its
// displacement d as d.(d + 2(p - r)) < 0, each bit flipped with probability
// floor(0.1 2^32) / 2^32.  A step draws its own five Philox calls (call index in bits 24-31
// of the second counter word); flags: bits 0-5 traits (1 = curious), 8-13 the true
// "came closer" bits, 16 terminal.
// ---------------------------------------------------------------------------------------
struct DrawCtx {                 // the counter words a self-drawing model step uses
  uint32_t k0, k1, purpose, c1;  // c1 = level | action << 8 | branch << 16
  unsigned long long node;
};

struct CrowdModel {
  static constexpr bool kStochastic = false;
  static constexpr bool kPairPacked = false;
  static constexpr bool kSelfDraw = true;
  static constexpr int kPeople = 6;
  struct S { float x, y; float px[6], py[6]; int f; };
  struct O { int o; };
  static constexpr uint32_t kReactThr = 3865470566u;   // floor(0.9 2^32)
  static constexpr uint32_t kFlipThr = 429496729u;     // floor(0.1 2^32)

  __device__ __forceinline__ static bool terminal(const S &s) { return (s.f >> 16) & 1; }
  __device__ __forceinline__ static uint4 words(const DrawCtx &c, uint32_t idx, uint32_t j) {
    return philox(make_uint4(c.c1 | (j << 24), idx | (c.purpose << 24), (uint32_t)c.node,
                             (uint32_t)(c.node >> 32)), c.k0, c.k1);
  }
  __device__ __forceinline__ static float step_drawn(S &s, int a, const DrawCtx &c, uint32_t idx) {
    if (terminal(s)) return 0.0f;
    uint4 w[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) w[j] = words(c, idx, (uint32_t)j);
    const float dxa = (a == 1) ? 1.0f : ((a == 3) ? -1.0f : 0.0f);
    const float dya = (a == 0) ? 1.0f : ((a == 2) ? -1.0f : 0.0f);
    const float nx = fminf(fmaxf(__fadd_rn(s.x, dxa), 0.0f), 50.0f);
    const float ny = fmaxf(__fadd_rn(s.y, dya), 0.0f);
    const bool exited = ny >= 40.0f;
    float r = (a == 4) ? -26.0f : -1.0f;
    const int traits = s.f & 0x3F;
    int closer = 0;
#pragma unroll
    for (int i = 0; i < kPeople; ++i) {
      // distances are compared squared; the direction uses one reciprocal square root
      const float ex = __fsub_rn(s.px[i], nx), ey = __fsub_rn(s.py[i], ny);
      const float q0 = fmaf(ex, ex, __fmul_rn(ey, ey));
      // the reaction (selects, not per-particle branches): YELL pushes a nearby person 2 m
      // away; otherwise with probability 0.9 a curious one steps toward the robot (at most
      // 0.3 m, never past it), a shy one 0.8 m away
      const bool near = q0 < 16.0f && q0 > 0.0f;
      const float inv = rsqrtf(near ? q0 : 1.0f);
      const float d0 = q0 * inv;
      const float ux = ex * inv, uy = ey * inv;
      const uint32_t wr = (i < 4) ? (&w[3].x)[i] : (&w[4].x)[i - 4];
      const bool react = near && (a == 4 || wr < kReactThr);
      const float sp = (a == 4) ? 2.0f : (((traits >> i) & 1) ? -fminf(d0, 0.3f) : 0.8f);
      const float mx = react ? sp * ux : 0.0f, my = react ? sp * uy : 0.0f;
      const uint4 wb = w[i >> 1];
      const float2 g = (i & 1) ? box_muller(wb.z, wb.w) : box_muller(wb.x, wb.y);
      const float ddx = fmaf(0.05f, g.x, mx), ddy = fmaf(0.05f, g.y, my);
      const float cl = fmaf(ddx, fmaf(2.0f, ex, ddx), __fmul_rn(ddy, fmaf(2.0f, ey, ddy)));
      if (cl < 0.0f) closer |= 1 << i;
      const float qx = fminf(fmaxf(__fadd_rn(s.px[i], ddx), 0.0f), 50.0f);
      const float qy = fminf(fmaxf(__fadd_rn(s.py[i], ddy), 0.0f), 40.0f);
      const float fx = __fsub_rn(qx, nx), fy = __fsub_rn(qy, ny);
      if (!exited && fmaf(fx, fx, __fmul_rn(fy, fy)) < 0.25f) r -= 200.0f;
      s.px[i] = qx;
      s.py[i] = qy;
    }
    s.x = nx;
    s.y = ny;
    s.f = traits | (closer << 8) | (exited ? (1 << 16) : 0);
    return exited ? r + 1000.0f : r;
  }
  // w0: the first observation call of counter (idx, c) (words 0, 1, 3 decide bits 0-2; word 2
  // picks a branch's representative); the second call decides bits 3-5.
  __device__ static O draw_obs_drawn(const S &s, const uint4 &w0, const DrawCtx &c, uint32_t idx) {
    const uint4 w1 = words(c, idx, 1u);
    const uint32_t u[6] = {w0.x, w0.y, w0.w, w1.x, w1.y, w1.z};
    int o = 0;
#pragma unroll
    for (int i = 0; i < kPeople; ++i) {
      int bit = (s.f >> (8 + i)) & 1;
      if (u[i] < kFlipThr) bit ^= 1;
      o |= bit << i;
    }
    return O{o};
  }
  __device__ __forceinline__ static O enum_obs(int k) { return O{k}; }
  // log2 Z(o | s') = sum over people of log2(1 - q) on agreement, log2 q otherwise
  __device__ __forceinline__ static float loglik2(const S &s, int, const O &o, const DevModel &) {
    if (o.o < 0 || o.o > 63) return -CUDART_INF_F;
    const int agree = 6 - __popc(((s.f >> 8) ^ o.o) & 0x3F);
    return (float)agree * -0.152003093f + (float)(6 - agree) * -3.32192809f;
  }
  // Z(o | s') = 2^(log2 Z), at least 2^-20 for a valid observation
  __device__ __forceinline__ static float zlin(const S &s, int a, const O &o, const DevModel &m) {
    return ex2(loglik2(s, a, o, m));
  }
  __device__ __forceinline__ static float loglik(const S &s, int a, const O &o, const DevModel &m) {
    return kLn2 * loglik2(s, a, o, m);
  }
  // h = a0 + b0 gamma^(m-1), m = max(1, 40 - y) unit moves north; 0 at terminal states
  __device__ __forceinline__ static float heuristic(const S &s, float log2g, float a0, float b0,
                                                    bool hz) {
    const float m = fmaxf(__fsub_rn(40.0f, s.y), 1.0f);
    const float h = fmaf(b0, ex2(fmaf(m, log2g, -log2g)), a0);
    return (hz || terminal(s)) ? 0.0f : h;
  }
  __device__ __forceinline__ static float heuristic(const S &s, const PlanDesc &P) {
    return heuristic(s, P.log2_gamma, P.h_a0, P.h_b0, P.h_zero != 0);
  }
  __device__ __forceinline__ static float2 obs_f2(const O &o) { return make_float2((float)o.o, 0.f); }
};

// Whether a model's step draws its own Philox calls (CROWD) or takes two words of the
// pair call of its particle (the others).
template <class M> struct SelfDraw { static constexpr bool value = false; };
template <> struct SelfDraw<CrowdModel> { static constexpr bool value = true; };

// Transition of particle i: from the pair words pw (words 0,1 for even i, 2,3 for odd i) or,
// for a self-drawing model, from its own calls under counter c with idx = i.
template <class M>
__device__ __forceinline__ float step_particle(typename M::S &s, int a, const uint4 &pw, int i,
                                              const DrawCtx &c, const DevModel &dm) {
  if constexpr (SelfDraw<M>::value) return M::step_drawn(s, a, c, (uint32_t)i);
  else return M::step(s, a, (i & 1) ? pw.z : pw.x, (i & 1) ? pw.w : pw.y, dm);
}
// Observation from the first observation call w of counter (idx, c) (and, for a
// self-drawing model, further calls of it).
template <class M>
__device__ __forceinline__ typename M::O obs_particle(const typename M::S &s, int a,
                                                      const uint4 &w, const DrawCtx &c,
                                                      uint32_t idx, const DevModel &dm) {
  if constexpr (SelfDraw<M>::value) return M::draw_obs_drawn(s, w, c, idx);
  else return M::draw_obs(s, a, w.x, w.y, dm);
}

}  // namespace vopp
