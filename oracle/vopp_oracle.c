/*
 * vopp_oracle.c -- plain, slow FP64 CPU oracle of the VOPP planning hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this file;
 * only the tests, the package's smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no source with the CUDA library: the Philox generator, the four models, the
 * tree recursion and the backup are all written out again here, in double precision, as
 * plain loops in the order the paper gives them.
 *
 * What it computes (VOPP, "Vectorized Online POMDP Planning"):
 *   - Eq. 1   V(b) = (1/eta_P) log sum_a exp(eta_P Psi(b,a))           (log-sum-exp value)
 *   - Eq. 2   Psi(b,a) = (1/eta_P) log pi0(a|b) + R(b,a) + gamma sum_o p(o|b,a) V(tau(b,a,o))
 *   - Eq. 3   one preference update from Psi_0 = (1/eta_P) log pi0 gives Psi_1 - L Psi_1 =
 *             log-softmax of (1/eta_P) log pi0 + Q, hence the closed form
 *             V(b) = eta * log sum_a pibar(a|b) exp(Q(b,a)/eta)  with eta = 1/eta_P.
 *   - Alg. 2  forward search: G(S,A) -> (S',O,R) per particle, leaf ValueHeuristic.
 *   - Alg. 3  backup: leaf value = aggregated heuristic; Q = mean reward + gamma * weighted
 *             mean child value (the action's total weight is the normaliser, Sec. III-E);
 *             V from the log-sum-exp over actions.
 *   - Alg. 1  root action = argmax_a Psi(root, a) = argmax_a Q(root,a) + eta log pibar(a).
 *   - Sec. III-B  belief update tau(b,a,o): sequential importance resampling.
 *
 * The tree is the full-width form: every action and W observation branches per action are
 * expanded at every node, each child carrying the whole weighted particle set.  Readings
 * where the paper is silent are fixed as follows (one place each, in this file):
 *   - eta here is the temperature (paper's eta_P = 1/eta).
 *   - SAMPLE branches: representative j uniform over particle indices, o_k ~ Z(.|s'_j,a),
 *     child weights w_i Z(o_k|s'_i), branch weight omega_k = N sum_i w_i Z_ik / sum_i Z_ik
 *     (importance ratio of the uniform-index proposal).  ENUMERATE branches: branch k is
 *     observation k and omega_k = p(o_k|b,a) = sum_i w_i Z_ik.
 *   - Q(b,a) = (1/W) sum_k rbar_k + gamma * sum_k omega_k V_k / sum_k omega_k, future 0 when
 *     sum_k omega_k = 0 (counted as degenerate).
 *   - terminal states are absorbing with reward 0 and heuristic 0.
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11) with the counter layout below.
 *
 * Counter layout (key = 64-bit seed, low word first):
 *   c0 = level | action << 8 | branch << 16, c1 = idx | purpose << 24, c2,c3 = node (lo,hi)
 *   purpose 0: transition noise of particle pair idx (words 0,1 -> particle 2idx, 2,3 -> 2idx+1)
 *   purpose 1: observation draw of a branch (words 0,1 -> noise / sense outcome, word 2 -> j)
 *   purpose 3: belief-update transition of pair idx, c0 = 0, node = time step t
 *   purpose 4: belief-update resampling offset, idx 0, c0 = 0, node = t
 *   purpose 5: environment transition of the true state, idx 0, c0 = 0, node = t
 *   purpose 6: environment observation, idx 0, c0 = 0, node = t (words 0,1 as purpose 1)
 *   episode mode (iteration k as the node word, episode e as idx, depth d as level):
 *   purpose 7: root state sample (word 0), 8: action sample (word 0), 9: transition
 *   (words 0,1), 10: observation (words 0,1)
 *   uniform:   u = (2 (x >> 9) + 1) * 2^-24, exactly representable in FP32 and FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXA 16
#define ORC_MAXD 8
#define ORC_MAXROCKS 8
#define ORC_MAXW 64

enum { ORC_NAV2D = 0, ORC_GRID = 1, ORC_TOY2 = 2, ORC_CROWD = 3 };
enum { ORC_SAMPLE = 0, ORC_ENUMERATE = 1 };
enum { ORC_PI_UNIFORM = 0, ORC_PI_FIXED = 1, ORC_PI_NAV_DIST = 2 };
enum { ORC_OK = 0, ORC_E_INVALID = -1, ORC_E_NOMEM = -2, ORC_E_DEGENERATE = -6 };

/* near-threshold band for the continuous goal test of NAV2D: |x^2 + y^2 - 0.25| < band */
#define ORC_NEAR_BAND 1e-5

typedef struct {
  int kind;          /* ORC_NAV2D / ORC_GRID / ORC_TOY2 */
  int branch_mode;   /* ORC_SAMPLE / ORC_ENUMERATE */
  int pi_mode;       /* ORC_PI_* */
  int h_zero;        /* 1: leaf heuristic forced to zero */
  double pi_temp;    /* temperature of the distance softmax (ORC_PI_NAV_DIST) */
  double pi_fixed[ORC_MAXA];
  int rock_x[ORC_MAXROCKS], rock_y[ORC_MAXROCKS];
} orc_model;

typedef struct {
  /* inputs */
  int N, D, W;
  double eta, gamma;
  uint64_t seed;
  int P;                   /* expand only path[0..P-1] at the top P levels (0 = whole tree) */
  int path[ORC_MAXD];      /* child slot a*W + k taken at each of the top P levels */
  int dump_levels;         /* dump particles of levels 0..dump_levels (-1 = none) */
  /* outputs (each may be NULL); level l spans n_l local nodes, concatenated by level */
  double *V;               /* [sum_l n_l]            node values, levels 0..D         */
  double *Q;               /* [sum_{l<D} n_l * A]    action values, levels 0..D-1     */
  double *rbar;            /* [sum_l n_l]            branch mean reward (level >= 1)  */
  double *lomega;          /* [sum_l n_l]            log branch weight (level >= 1)   */
  double *obs;             /* [sum_l n_l * 2]        branch observation               */
  int32_t *rep;            /* [sum_l n_l]            representative index j           */
  uint8_t *near;           /* [sum_l n_l]            near-threshold event at creation */
  double *px, *py, *plw;   /* [sum_{l<=dump} n_l * N] particle dumps (NAV2D x,y; lw)  */
  int32_t *ps;             /* [sum_{l<=dump} n_l * N] particle dumps (GRID / TOY2)    */
  /* results */
  int action;
  double v_root;
  double q_root[ORC_MAXA];
  double policy[ORC_MAXA];
  long long near_threshold, degenerate, particle_steps;
  /* anytime iterative deepening (Alg. 1 loop, Eq. 3): when psi is set, every internal node
   * keeps its preferences Psi(n, .) in psi[(off_l + n) * A + a] across calls, and the backup
   * updates them instead of using the one-pass closed form.  Nodes at levels >=
   * psi_new_level start from Psi_0 = eta log pibar. */
  double *psi;             /* [sum_{l<D} n_l * A] or NULL                                   */
  int psi_new_level;
  /* CROWD: root people coordinates [12][N] (px_q = row 2q, py_q = row 2q + 1); dumps of the
   * people coordinates [sum_{l<=dump} n_l][12][N] (robot in px/py, flags in ps) */
  const double *root_pf;
  double *ppf;
} orc_plan_args;

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 products */
/* with the Weyl key schedule.                                                             */
/* ------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)0xD2511F53u * x0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ x1 ^ k0;
    uint32_t n2 = hi0 ^ x3 ^ k1;
    x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw_j(uint64_t seed, uint32_t idx, uint32_t purpose, uint32_t level, uint32_t action,
                   uint32_t branch, uint32_t call, uint64_t node, uint32_t out[4]) {
  uint32_t ctr[4], key[2];
  ctr[0] = level | (action << 8) | (branch << 16) | (call << 24);
  ctr[1] = idx | (purpose << 24);
  ctr[2] = (uint32_t)node;
  ctr[3] = (uint32_t)(node >> 32);
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32);
  orc_philox4x32_10(ctr, key, out);
}

static void draw(uint64_t seed, uint32_t idx, uint32_t purpose, uint32_t level, uint32_t action,
                 uint32_t branch, uint64_t node, uint32_t out[4]) {
  draw_j(seed, idx, purpose, level, action, branch, 0, node, out);
}

double orc_uniform(uint32_t x) { return (2.0 * (double)(x >> 9) + 1.0) * (1.0 / 16777216.0); }

/* Box-Muller: two independent N(0,1) from two uniforms. */
void orc_box_muller(uint32_t a, uint32_t b, double *g1, double *g2) {
  double u1 = orc_uniform(a), u2 = orc_uniform(b);
  double r = sqrt(-2.0 * log(u1));
  *g1 = r * cos(2.0 * M_PI * u2);
  *g2 = r * sin(2.0 * M_PI * u2);
}

static double lse_pair_max(double m, double v) { return v > m ? v : m; }

/* log sum_i exp(v_i), -inf when every term is -inf (Eq. 1's log-sum-exp operator). */
static double log_sum_exp(const double *v, int n) {
  double m = -INFINITY;
  for (int i = 0; i < n; ++i) m = lse_pair_max(m, v[i]);
  if (m == -INFINITY) return -INFINITY;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += exp(v[i] - m);
  return m + log(s);
}

/* ------------------------------------------------------------------------------------ */
/* The three generative models G(s,a) -> (s', o, r) (Sec. III-B).                         */
/* ------------------------------------------------------------------------------------ */
int orc_num_actions(int kind) {
  return kind == ORC_NAV2D ? 4 : kind == ORC_GRID ? 13 : kind == ORC_CROWD ? 5 : 2;
}
static int num_obs(int kind) {
  return kind == ORC_NAV2D ? 0 : kind == ORC_GRID ? 3 : kind == ORC_CROWD ? 64 : 2;
}

/* particle state: NAV2D (x, y); GRID / TOY2 s; CROWD robot (x, y), people (px, py), s = flags */
#define CR_N 6
typedef struct { double x, y; int32_t s; double px[CR_N], py[CR_N]; } pstate;

/* Counter of a particle's random numbers (CROWD draws several Philox calls per step; call j
 * sits in bits 24-31 of the second counter word, which the other models leave 0). */
typedef struct { uint64_t seed; uint32_t idx, purpose, level, action, branch; uint64_t node; } orc_ctr;

/* NAV2D: (x,y) in [0,10]^2, goal disc of radius 0.5 at the origin is absorbing. */
static const double NAV_DX[4] = {1.0, -1.0, 0.0, 0.0};
static const double NAV_DY[4] = {0.0, 0.0, 1.0, -1.0};
static int nav_terminal(double x, double y) { return x * x + y * y <= 0.25; }
static int nav_near(double x, double y) { return fabs(x * x + y * y - 0.25) < ORC_NEAR_BAND; }
static double clamp10(double v) { return v < 0.0 ? 0.0 : (v > 10.0 ? 10.0 : v); }
static double nav_sigma(double x) { return 0.5 * fabs(x - 9.0) + 0.05; }

/* GRIDSENSE: packed state, bits 0-7 rocks, 8-11 x (11 = exited), 12-15 y, 16 terminal. */
#define G_X(s) (((s) >> 8) & 0xF)
#define G_Y(s) (((s) >> 12) & 0xF)
#define G_TERM(s) (((s) >> 16) & 1)
static int32_t g_pack(int32_t rocks, int x, int y, int term) {
  return (rocks & 0xFF) | (x << 8) | (y << 12) | (term << 16);
}

/* sense accuracy 0.5 + 0.5 exp(-d/4), d the Euclidean agent-rock distance */
double orc_grid_acc(int d2) { return 0.5 + 0.5 * exp(-sqrt((double)d2) / 4.0); }

/* sense outcome is correct iff a Philox word u satisfies u < floor(acc * 2^32) */
uint64_t orc_grid_threshold(int d2) { return (uint64_t)floor(orc_grid_acc(d2) * 4294967296.0); }

static int rock_at(const orc_model *m, int x, int y) {
  for (int r = 0; r < ORC_MAXROCKS; ++r)
    if (m->rock_x[r] == x && m->rock_y[r] == y) return r;
  return -1;
}

static int grid_d2(const orc_model *m, int32_t s, int rock) {
  int dx = G_X(s) - m->rock_x[rock], dy = G_Y(s) - m->rock_y[rock];
  return dx * dx + dy * dy;
}

/* CROWD (Sec. IV, CrowdNav): a robot in a 50 x 40 m hall and the CR_N nearest people, each
 * curious or shy (hidden).  Actions 0 NORTH, 1 EAST, 2 SOUTH, 3 WEST (1 m), 4 YELL.  Every
 * person moves by N(0, 0.05^2) noise per axis; a person within 4 m of the robot's new
 * position reacts with probability 0.9 -- curious toward it by 0.3 m (never past it), shy
 * away by 0.8 m -- and under YELL every such person backs away by 2 m instead.  People stay
 * in the hall; the robot is held by the east, west and south walls and leaves through the
 * north border (y >= 40: +1000, terminal).  Reward -1 per step, -25 for YELL, -200 per
 * person within 0.5 m after the step.  Observation: per person, whether the distance to
 * the robot's new position decreased -- taken from the person's displacement d as
 * d.(d + 2(p - r)) < 0, which is that comparison away from the walls and stays the same in
 * FP32 and FP64 except within 1e-7 of a tie -- each bit flipped with probability
 * q = floor(0.1 2^32) / 2^32.  Near-threshold events (reaction radius, bump radius, closer
 * ties) are counted like NAV2D's goal test.  Flags: bits 0-5 traits (1 = curious), 8-13 the true "came closer" bits, 16
 * terminal. */
#define CR_W 50.0
#define CR_H 40.0
#define CR_RNEAR 4.0
#define CR_VCUR 0.3
#define CR_VSHY 0.8
#define CR_VBACK 2.0
#define CR_SIGP 0.05
#define CR_RBUMP 0.5
static const double CR_DX[5] = {0.0, 1.0, 0.0, -1.0, 0.0};
static const double CR_DY[5] = {1.0, 0.0, -1.0, 0.0, 0.0};
static const uint32_t CR_REACT_THR = 3865470566u;   /* floor(0.9 * 2^32) */
static const uint32_t CR_FLIP_THR = 429496729u;     /* floor(0.1 * 2^32) */
#define CR_TERM(s) (((s) >> 16) & 1)

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void crowd_step(const pstate *in, int a, const orc_ctr *c, pstate *out, double *reward,
                       long long *near) {
  *out = *in;
  if (CR_TERM(in->s)) { *reward = 0.0; return; }
  uint32_t w[5][4];
  for (uint32_t j = 0; j < 5; ++j)
    draw_j(c->seed, c->idx, c->purpose, c->level, c->action, c->branch, j, c->node, w[j]);
  double r = -1.0 + (a == 4 ? -25.0 : 0.0);
  const double nx = clampd(in->x + CR_DX[a], 0.0, CR_W), ny = in->y + CR_DY[a] < 0.0 ? 0.0 : in->y + CR_DY[a];
  out->x = nx;
  out->y = ny;
  const int traits = in->s & 0x3F;
  int closer = 0;
  const int exited = ny >= CR_H;
  for (int i = 0; i < CR_N; ++i) {
    const double px = in->px[i], py = in->py[i];
    const double ex = px - nx, ey = py - ny;        /* robot (new position) to the person */
    const double d0 = sqrt(ex * ex + ey * ey);
    double mx = 0.0, my = 0.0;                       /* the person's reaction */
    if (d0 < CR_RNEAR && d0 > 0.0) {
      const double ux = ex / d0, uy = ey / d0;       /* away from the robot */
      const uint32_t wr = i < 4 ? w[3][i] : w[4][i - 4];
      if (a == 4) {
        mx = CR_VBACK * ux; my = CR_VBACK * uy;
      } else if (wr < CR_REACT_THR) {
        if ((traits >> i) & 1) {
          const double st = d0 < CR_VCUR ? d0 : CR_VCUR;
          mx = -st * ux; my = -st * uy;
        } else {
          mx = CR_VSHY * ux; my = CR_VSHY * uy;
        }
      }
    }
    if (fabs(d0 - CR_RNEAR) < 1e-4) ++*near;
    double g1, g2;
    orc_box_muller(w[i / 2][2 * (i % 2)], w[i / 2][2 * (i % 2) + 1], &g1, &g2);
    const double dx = mx + CR_SIGP * g1, dy = my + CR_SIGP * g2;   /* displacement */
    /* came closer: |p + d - r| < |p - r|, i.e. d.(d + 2(p - r)) < 0 (from the displacement,
     * before the walls clamp the position) */
    const double cl = dx * (dx + 2.0 * ex) + dy * (dy + 2.0 * ey);
    if (cl < 0.0) closer |= 1 << i;
    if (fabs(cl) < 1e-7) ++*near;
    const double qx = clampd(px + dx, 0.0, CR_W), qy = clampd(py + dy, 0.0, CR_H);
    const double d1 = hypot(qx - nx, qy - ny);
    if (!exited && d1 < CR_RBUMP) r -= 200.0;
    if (!exited && fabs(d1 - CR_RBUMP) < 1e-4) ++*near;
    out->px[i] = qx;
    out->py[i] = qy;
  }
  if (exited) r += 1000.0;
  out->s = traits | (closer << 8) | (exited << 16);
  *reward = r;
}

/* observation bits: word k of the branch's calls decides the flip of bit k */
static int crowd_draw_obs(const pstate *sp, const orc_ctr *c) {
  uint32_t w0[4], w1[4];
  draw_j(c->seed, c->idx, c->purpose, c->level, c->action, c->branch, 0, c->node, w0);
  draw_j(c->seed, c->idx, c->purpose, c->level, c->action, c->branch, 1, c->node, w1);
  const uint32_t u[CR_N] = {w0[0], w0[1], w0[3], w1[0], w1[1], w1[2]};
  int o = 0;
  for (int i = 0; i < CR_N; ++i) {
    int bit = (sp->s >> (8 + i)) & 1;
    if (u[i] < CR_FLIP_THR) bit ^= 1;
    o |= bit << i;
  }
  return o;
}

static double crowd_loglik(const pstate *sp, int o) {
  const double q = (double)CR_FLIP_THR / 4294967296.0;
  double l = 0.0;
  for (int i = 0; i < CR_N; ++i)
    l += (((sp->s >> (8 + i)) & 1) == ((o >> i) & 1)) ? log(1.0 - q) : log(q);
  return l;
}

/* One transition step.  wa, wb: the two Philox words of this particle (NAV2D); c: the
 * counter of the particle's own calls (CROWD). */
static void model_step(const orc_model *m, const pstate *in, int a, uint32_t wa, uint32_t wb,
                       const orc_ctr *c, pstate *out, double *reward, long long *near) {
  if (m->kind == ORC_CROWD) {
    crowd_step(in, a, c, out, reward, near);
    return;
  }
  if (m->kind == ORC_NAV2D) {
    if (nav_terminal(in->x, in->y)) { *out = *in; *reward = 0.0; return; }
    double g1, g2;
    orc_box_muller(wa, wb, &g1, &g2);
    out->x = clamp10(in->x + NAV_DX[a] + 0.1 * g1);
    out->y = clamp10(in->y + NAV_DY[a] + 0.1 * g2);
    out->s = 0;
    *reward = nav_terminal(out->x, out->y) ? 100.0 : -1.0;
    if (nav_near(out->x, out->y)) ++*near;
  } else if (m->kind == ORC_GRID) {
    int32_t s = in->s;
    out->x = out->y = 0.0;
    if (G_TERM(s)) { out->s = s; *reward = 0.0; return; }
    int x = G_X(s), y = G_Y(s), rocks = s & 0xFF;
    *reward = 0.0;
    if (a == 0) {                       /* east: leaving the grid ends the episode, +10 */
      if (x == 10) { out->s = g_pack(rocks, 11, y, 1); *reward = 10.0; return; }
      x += 1;
    } else if (a == 1) { if (x > 0) x -= 1; }      /* west */
    else if (a == 2) { if (y < 10) y += 1; }       /* north */
    else if (a == 3) { if (y > 0) y -= 1; }        /* south */
    else if (a == 4) {                              /* collect */
      int r = rock_at(m, x, y);
      if (r >= 0) {
        if ((rocks >> r) & 1) { *reward = 10.0; rocks &= ~(1 << r); }
        else *reward = -10.0;
      }
    }                                               /* a >= 5: sense, state unchanged */
    out->s = g_pack(rocks, x, y, 0);
  } else {                                          /* TOY2: 0 = stay, 1 = flip */
    int32_t s = in->s;
    out->x = out->y = 0.0;
    out->s = (a == 1) ? 1 - s : s;
    *reward = (a == 1) ? -0.1 : (s == 0 ? 1.0 : -1.0);
  }
}

/* o ~ Z(. | s', a) drawn with Philox words (w0,w1).  NAV2D fills o[0..1]; discrete models
 * store the observation index in o[0]. */
static void model_draw_obs(const orc_model *m, const pstate *sp, int a, uint32_t w0, uint32_t w1,
                           const orc_ctr *c, double o[2]) {
  if (m->kind == ORC_CROWD) {
    o[0] = (double)crowd_draw_obs(sp, c);
    o[1] = 0.0;
    return;
  }
  if (m->kind == ORC_NAV2D) {
    double g3, g4, sg = nav_sigma(sp->x);
    orc_box_muller(w0, w1, &g3, &g4);
    o[0] = sp->x + sg * g3;
    o[1] = sp->y + sg * g4;
  } else if (m->kind == ORC_GRID) {
    o[1] = 0.0;
    if (a < 5) { o[0] = 0.0; return; }               /* NULL observation */
    int r = a - 5, bit = (sp->s >> r) & 1;
    int correct = (uint64_t)w0 < orc_grid_threshold(grid_d2(m, sp->s, r));
    int seen = correct ? bit : 1 - bit;
    o[0] = seen ? 1.0 : 2.0;                        /* 1 = good, 2 = bad */
  } else {
    int correct = (uint64_t)w0 < (uint64_t)floor(0.85 * 4294967296.0);
    o[0] = correct ? sp->s : 1 - sp->s;
    o[1] = 0.0;
  }
}

/* log Z(o | s', a); -inf where the observation is impossible. */
static double model_loglik(const orc_model *m, const pstate *sp, int a, const double o[2]) {
  if (m->kind == ORC_CROWD) {
    const int oi = (int)o[0];
    if (oi < 0 || oi > 63) return -INFINITY;
    return crowd_loglik(sp, oi);
  }
  if (m->kind == ORC_NAV2D) {
    double sg = nav_sigma(sp->x);
    double dx = o[0] - sp->x, dy = o[1] - sp->y;
    return -(dx * dx + dy * dy) / (2.0 * sg * sg) - 2.0 * log(sg) - log(2.0 * M_PI);
  } else if (m->kind == ORC_GRID) {
    int oi = (int)o[0];
    if (a < 5) return oi == 0 ? 0.0 : -INFINITY;
    if (oi == 0) return -INFINITY;
    int r = a - 5, bit = (sp->s >> r) & 1;
    double acc = orc_grid_acc(grid_d2(m, sp->s, r));
    int seen = (oi == 1);
    return seen == bit ? log(acc) : log(1.0 - acc);
  } else {
    int oi = (int)o[0];
    if (oi < 0 || oi > 1) return -INFINITY;        /* only observations 0 and 1 exist */
    return (oi == sp->s) ? log(0.85) : log(0.15);
  }
}

/* Leaf ValueHeuristic (Alg. 2): optimistic discounted return to the goal / exit. */
static double model_heuristic(const orc_model *m, const pstate *s, double gamma) {
  if (m->h_zero) return 0.0;
  if (m->kind == ORC_NAV2D) {
    if (nav_terminal(s->x, s->y)) return 0.0;
    double steps = s->x + s->y - 0.5;          /* unit moves to the goal disc (continuous) */
    if (steps < 1.0) steps = 1.0;
    double gk = pow(gamma, steps - 1.0);
    /* -1 for each of the first steps-1 moves, then +100 on arrival */
    return -(1.0 - gk) / (1.0 - gamma) + 100.0 * gk;
  } else if (m->kind == ORC_GRID) {
    if (G_TERM(s->s)) return 0.0;
    return 10.0 * pow(gamma, (double)(10 - G_X(s->s)));
  } else if (m->kind == ORC_CROWD) {
    if (CR_TERM(s->s)) return 0.0;
    double steps = CR_H - s->y;              /* 1 m moves north to the border (continuous) */
    if (steps < 1.0) steps = 1.0;
    double gk = pow(gamma, steps - 1.0);
    return -(1.0 - gk) / (1.0 - gamma) + 1000.0 * gk;
  }
  return 0.0;
}

static int model_is_terminal(const orc_model *m, const pstate *s) {
  if (m->kind == ORC_NAV2D) return nav_terminal(s->x, s->y);
  if (m->kind == ORC_GRID) return G_TERM(s->s);
  if (m->kind == ORC_CROWD) return CR_TERM(s->s);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Reference policy pibar(a|b) (Sec. III-A): uniform, a fixed vector, or a softmax of the   */
/* negative distance-to-goal of the weighted mean particle after each action.               */
/* ------------------------------------------------------------------------------------ */
static void log_pibar(const orc_model *m, const pstate *p, const double *lw, int N, double *out) {
  int A = orc_num_actions(m->kind);
  if (m->pi_mode == ORC_PI_UNIFORM) {
    for (int a = 0; a < A; ++a) out[a] = -log((double)A);
    return;
  }
  double z[ORC_MAXA] = {0};
  if (m->pi_mode == ORC_PI_FIXED) {
    for (int a = 0; a < A; ++a) z[a] = m->pi_fixed[a] > 0.0 ? log(m->pi_fixed[a]) : -INFINITY;
  } else {
    double mx = 0.0, my = 0.0;
    for (int i = 0; i < N; ++i) { double w = exp(lw[i]); mx += w * p[i].x; my += w * p[i].y; }
    for (int a = 0; a < A; ++a) {
      double cx = clamp10(mx + NAV_DX[a]), cy = clamp10(my + NAV_DY[a]);
      z[a] = -sqrt(cx * cx + cy * cy) / m->pi_temp;
    }
  }
  double lz = log_sum_exp(z, A);
  for (int a = 0; a < A; ++a) out[a] = z[a] - lz;
}

/* V(b) = eta * log sum_a pibar(a|b) exp(Q(b,a)/eta)   (Eq. 1 after one Eq. 3 update) */
static double belief_value(const double *q, const double *lpi, int A, double eta) {
  double z[ORC_MAXA] = {0};
  for (int a = 0; a < A; ++a) z[a] = lpi[a] + q[a] / eta;
  return eta * log_sum_exp(z, A);
}

/* [L_eta Psi](b) = eta * log sum_a exp(Psi(b,a)/eta)   (Eq. 1 with the temperature eta) */
static double lse_value(const double *psi, int A, double eta) {
  double z[ORC_MAXA] = {0};
  for (int a = 0; a < A; ++a) z[a] = psi[a] / eta;
  return eta * log_sum_exp(z, A);
}

/* One preference update of a node (Eq. 3; Alg. 3 steps V_curr, Psi update, V):
 *   V_curr = L Psi;  Psi <- Psi - V_curr + Q;  returns V = L Psi.
 * A node that has no preferences yet starts from Psi_0 = eta log pibar. */
static double preference_update(double *psi, const double *q, const double *lpi, int fresh,
                                int A, double eta) {
  if (fresh)
    for (int a = 0; a < A; ++a) psi[a] = eta * lpi[a];
  double vcur = lse_value(psi, A, eta);
  for (int a = 0; a < A; ++a) psi[a] = psi[a] - vcur + q[a];
  return lse_value(psi, A, eta);
}

/* ------------------------------------------------------------------------------------ */
/* Full-width tree recursion (Alg. 2 forward search, Alg. 3 backup), depth first.          */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  const orc_model *m;
  orc_plan_args *io;
  int A, W, AW, N, D, P;
  long long off[ORC_MAXD + 2];      /* level offsets into the concatenated outputs */
  pstate *lev[ORC_MAXD + 1];        /* particle states per level                   */
  double *lw[ORC_MAXD + 1];         /* normalised log weights per level            */
  double *ell, *tmp, *rew;
} orc_tree;

static long long level_size(int l, int P, int AW) {
  long long n = 1;
  for (int i = P; i < l; ++i) n *= AW;
  return n;
}

static void dump_particles(orc_tree *t, int l, long long lnode) {
  orc_plan_args *io = t->io;
  if (l > io->dump_levels) return;
  long long base = (t->off[l] + lnode) * t->N;
  for (int i = 0; i < t->N; ++i) {
    if (io->px) io->px[base + i] = t->lev[l][i].x;
    if (io->py) io->py[base + i] = t->lev[l][i].y;
    if (io->ps) io->ps[base + i] = t->lev[l][i].s;
    if (io->plw) io->plw[base + i] = t->lw[l][i];
    if (io->ppf)
      for (int q = 0; q < CR_N; ++q) {
        io->ppf[(base * 12) + (2 * q) * t->N + i] = t->lev[l][i].px[q];
        io->ppf[(base * 12) + (2 * q + 1) * t->N + i] = t->lev[l][i].py[q];
      }
  }
}

/* Build child (a,k) of node gnode at level l into level l+1 (G, observation, weighting). */
static void make_child(orc_tree *t, int l, uint64_t gnode, int a, int k, long long cl,
                       double *rbar_out, double *lomega_out) {
  const orc_model *m = t->m;
  orc_plan_args *io = t->io;
  int N = t->N;
  pstate *par = t->lev[l], *ch = t->lev[l + 1];
  double *plw = t->lw[l], *clw = t->lw[l + 1];
  long long near = 0;

  /* G(S, A): every particle steps under action a with this branch's own noise */
  for (int i = 0; i < N; ++i) {
    uint32_t w[4] = {0, 0, 0, 0};
    if (m->kind == ORC_NAV2D) draw(io->seed, (uint32_t)(i / 2), 0, l, a, k, gnode, w);
    uint32_t wa = (i & 1) ? w[2] : w[0], wb = (i & 1) ? w[3] : w[1];
    const orc_ctr c = {io->seed, (uint32_t)i, 0, (uint32_t)l, (uint32_t)a, (uint32_t)k, gnode};
    model_step(m, &par[i], a, wa, wb, &c, &ch[i], &t->rew[i], &near);
  }
  io->particle_steps += N;

  /* the branch observation */
  double o[2];
  int j = -1;
  if (m->branch_mode == ORC_SAMPLE) {
    uint32_t w[4];
    draw(io->seed, 0, 1, l, a, k, gnode, w);
    j = (int)(((uint64_t)w[2] * (uint64_t)N) >> 32);
    const orc_ctr c = {io->seed, 0, 1, (uint32_t)l, (uint32_t)a, (uint32_t)k, gnode};
    model_draw_obs(m, &ch[j], a, w[0], w[1], &c, o);
  } else {
    o[0] = (double)k;
    o[1] = 0.0;
  }

  /* log-likelihoods, reward mean, weights */
  double rbar = 0.0;
  for (int i = 0; i < N; ++i) {
    t->ell[i] = model_loglik(m, &ch[i], a, o);
    t->tmp[i] = plw[i] + t->ell[i];
    rbar += exp(plw[i]) * t->rew[i];
  }
  double ls1 = log_sum_exp(t->tmp, N);
  double lomega;
  if (m->branch_mode == ORC_SAMPLE) {
    double ls0 = log_sum_exp(t->ell, N);
    lomega = (ls1 == -INFINITY) ? -INFINITY : log((double)N) + ls1 - ls0;
  } else {
    lomega = ls1;
  }
  for (int i = 0; i < N; ++i) clw[i] = (ls1 == -INFINITY) ? -INFINITY : t->tmp[i] - ls1;

  long long idx = t->off[l + 1] + cl;
  if (io->rbar) io->rbar[idx] = rbar;
  if (io->lomega) io->lomega[idx] = lomega;
  if (io->rep) io->rep[idx] = j;
  if (io->obs) { io->obs[2 * idx] = o[0]; io->obs[2 * idx + 1] = o[1]; }
  if (io->near) io->near[idx] = (uint8_t)(near > 0);
  io->near_threshold += near;
  *rbar_out = rbar;
  *lomega_out = lomega;
}

static double expand(orc_tree *t, int l, uint64_t gnode, long long lnode) {
  const orc_model *m = t->m;
  orc_plan_args *io = t->io;
  int N = t->N, A = t->A, W = t->W;
  dump_particles(t, l, lnode);

  if (l == t->D) {                          /* leaf: weighted mean of the heuristic */
    double v = 0.0;
    for (int i = 0; i < N; ++i) v += exp(t->lw[l][i]) * model_heuristic(m, &t->lev[l][i], io->gamma);
    if (io->V) io->V[t->off[l] + lnode] = v;
    return v;
  }

  double lpi[ORC_MAXA];
  log_pibar(m, t->lev[l], t->lw[l], N, lpi);

  double rb[ORC_MAXA][ORC_MAXW], lom[ORC_MAXA][ORC_MAXW], vc[ORC_MAXA][ORC_MAXW];
  int on_path = l < t->P;
  for (int a = 0; a < A; ++a) {
    for (int k = 0; k < W; ++k) {
      int slot = a * W + k;
      if (on_path && slot != io->path[l]) continue;
      uint64_t cg = gnode * (uint64_t)t->AW + (uint64_t)slot;
      long long cl = (l + 1 <= t->P) ? 0 : lnode * t->AW + slot;
      make_child(t, l, gnode, a, k, cl, &rb[a][k], &lom[a][k]);
      vc[a][k] = expand(t, l + 1, cg, cl);
    }
  }
  if (on_path) return NAN;                 /* partial node: only one child expanded */

  /* Alg. 3: Q = mean reward + gamma * omega-weighted mean of child values */
  double q[ORC_MAXA] = {0};
  for (int a = 0; a < A; ++a) {
    double rsum = 0.0, mx = -INFINITY;
    for (int k = 0; k < W; ++k) { rsum += rb[a][k]; if (lom[a][k] > mx) mx = lom[a][k]; }
    double fut = 0.0;
    if (mx == -INFINITY) {
      ++io->degenerate;
    } else {
      double num = 0.0, den = 0.0;
      for (int k = 0; k < W; ++k) {
        double om = exp(lom[a][k] - mx);
        num += om * vc[a][k];
        den += om;
      }
      fut = num / den;
    }
    q[a] = rsum / W + io->gamma * fut;
  }
  /* Psi of this node: one-pass closed form, or the persistent preferences (anytime mode) */
  double ps[ORC_MAXA];
  double v;
  if (io->psi) {
    double *pn = io->psi + (t->off[l] + lnode) * A;
    v = preference_update(pn, q, lpi, l >= io->psi_new_level, A, io->eta);
    for (int a = 0; a < A; ++a) ps[a] = pn[a];
  } else {
    v = belief_value(q, lpi, A, io->eta);
    for (int a = 0; a < A; ++a) ps[a] = q[a] + io->eta * lpi[a];
  }
  if (io->Q) for (int a = 0; a < A; ++a) io->Q[(t->off[l] + lnode) * A + a] = q[a];
  if (io->V) io->V[t->off[l] + lnode] = v;

  if (l == 0) {                             /* Alg. 1: root action = argmax Psi */
    int best = 0;
    double bs = -INFINITY;
    for (int a = 0; a < A; ++a) {
      if (ps[a] > bs) { bs = ps[a]; best = a; }
      io->q_root[a] = q[a];
      io->policy[a] = exp((ps[a] - v) / io->eta);
    }
    io->action = best;
    io->v_root = v;
  }
  return v;
}

/* Root preparation: normalise caller weights, zero particles already terminal. */
static int root_prep(const orc_model *m, const pstate *root, const double *w, int N, pstate *dst,
                     double *lw, long long *near) {
  double tot = 0.0;
  for (int i = 0; i < N; ++i) {
    dst[i] = root[i];
    double wi = w ? w[i] : 1.0;
    if (wi < 0.0) return ORC_E_INVALID;
    if (model_is_terminal(m, &root[i])) wi = 0.0;
    if (m->kind == ORC_NAV2D && nav_near(root[i].x, root[i].y)) ++*near;
    lw[i] = wi;
    tot += wi;
  }
  if (!(tot > 0.0)) return ORC_E_DEGENERATE;
  for (int i = 0; i < N; ++i) lw[i] = lw[i] > 0.0 ? log(lw[i] / tot) : -INFINITY;
  return ORC_OK;
}

/* Level offsets of the concatenated per-level outputs. */
void orc_level_offsets(int A, int W, int D, int P, long long *off) {
  off[0] = 0;
  for (int l = 0; l <= D; ++l) off[l + 1] = off[l] + level_size(l, P, A * W);
}

/*
 * One plan (Alg. 1 with a single full-width search episode and one backup pass).
 * root_x/root_y: NAV2D particle coordinates (CROWD robot); root_s: GRID/TOY2 states (CROWD
 * flags; people in io->root_pf); root_w: weights or
 * NULL for uniform.  Returns ORC_OK, ORC_E_INVALID, ORC_E_NOMEM or ORC_E_DEGENERATE.
 */
int orc_plan(const orc_model *m, const double *root_x, const double *root_y,
             const int32_t *root_s, const double *root_w, orc_plan_args *io) {
  orc_tree t;
  memset(&t, 0, sizeof t);
  t.m = m;
  t.io = io;
  t.A = orc_num_actions(m->kind);
  t.W = io->W;
  t.AW = t.A * t.W;
  t.N = io->N;
  t.D = io->D;
  t.P = io->P;
  if (t.N < 1 || t.D < 0 || t.D > ORC_MAXD || t.W < 1 || t.W > ORC_MAXW || t.P < 0 || t.P > t.D || !(io->eta > 0.0) || !(io->gamma > 0.0) ||
      !(io->gamma < 1.0))
    return ORC_E_INVALID;
  if (m->branch_mode == ORC_ENUMERATE && (m->kind == ORC_NAV2D || t.W < num_obs(m->kind)))
    return ORC_E_INVALID;
  for (int l = 0; l < t.P; ++l)
    if (io->path[l] < 0 || io->path[l] >= t.AW) return ORC_E_INVALID;
  if (io->psi && (t.P > 0 || t.D < 1)) return ORC_E_INVALID;   /* anytime: whole trees, D >= 1 */
  orc_level_offsets(t.A, t.W, t.D, t.P, t.off);
  io->near_threshold = io->degenerate = io->particle_steps = 0;
  io->action = -1;
  io->v_root = NAN;

  int rc = ORC_OK;
  for (int l = 0; l <= t.D; ++l) {
    t.lev[l] = (pstate *)calloc((size_t)t.N, sizeof(pstate));
    t.lw[l] = (double *)calloc((size_t)t.N, sizeof(double));
    if (!t.lev[l] || !t.lw[l]) rc = ORC_E_NOMEM;
  }
  t.ell = (double *)calloc((size_t)t.N, sizeof(double));
  t.tmp = (double *)calloc((size_t)t.N, sizeof(double));
  t.rew = (double *)calloc((size_t)t.N, sizeof(double));
  pstate *root = (pstate *)calloc((size_t)t.N, sizeof(pstate));
  if (!t.ell || !t.tmp || !t.rew || !root) rc = ORC_E_NOMEM;

  if (rc == ORC_OK) {
    for (int i = 0; i < t.N; ++i) {
      root[i].x = root_x ? root_x[i] : 0.0;
      root[i].y = root_y ? root_y[i] : 0.0;
      root[i].s = root_s ? root_s[i] : 0;
      if (io->root_pf)
        for (int q = 0; q < CR_N; ++q) {
          root[i].px[q] = io->root_pf[(2 * q) * t.N + i];
          root[i].py[q] = io->root_pf[(2 * q + 1) * t.N + i];
        }
    }
    long long near = 0;
    rc = root_prep(m, root, root_w, t.N, t.lev[0], t.lw[0], &near);
    io->near_threshold += near;
  }
  if (rc == ORC_OK) {
    /* with P > 0 the recursion walks down the path with single-child expansions and then
     * expands the whole subtree below the path node */
    if (t.P == 0) {
      if (t.D == 0) {
        /* depth 0: V = mean heuristic, every Q equal to it, action = argmax pibar */
        double lpi[ORC_MAXA];
        double v = expand(&t, 0, 0, 0);
        log_pibar(m, t.lev[0], t.lw[0], t.N, lpi);
        int best = 0;
        for (int a = 0; a < t.A; ++a) {
          io->q_root[a] = v;
          io->policy[a] = exp(lpi[a]);
          if (lpi[a] > lpi[best]) best = a;
          if (io->Q) io->Q[a] = v;
        }
        io->action = best;
        io->v_root = v;
      } else {
        expand(&t, 0, 0, 0);
      }
    } else {
      expand(&t, 0, 0, 0);
    }
  }
  for (int l = 0; l <= t.D; ++l) { free(t.lev[l]); free(t.lw[l]); }
  free(t.ell); free(t.tmp); free(t.rew); free(root);
  return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Belief update tau(b,a,o): sequential importance resampling (Sec. III-B).               */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  double ess;
  int resampled;
  int ess_tie;               /* ESS within 1e-4 N of the resampling threshold N/2 */
  long long near_ties;
  uint8_t *ties;             /* optional [N]: output position within 1e-5 of a CDF boundary */
  double *prop_x, *prop_y;   /* optional [N]: propagated states before resampling */
  int32_t *prop_s;
  double *pf;                /* CROWD people coordinates [12][N] (px_q = row 2q, py_q = 2q+1),
                                updated like x, y, s; NULL for the other models */
} orc_bu_result;

int orc_belief_update(const orc_model *m, int N, double *x, double *y, int32_t *s, double *lw,
                      int action, const double *obs, uint64_t seed, uint64_t t_step,
                      int32_t *ancestors, orc_bu_result *res) {
  double *pf = res->pf;
  if (N < 1 || action < 0 || action >= orc_num_actions(m->kind)) return ORC_E_INVALID;
  pstate *sp = (pstate *)calloc((size_t)N, sizeof(pstate));
  double *nl = (double *)calloc((size_t)N, sizeof(double));
  double *cdf = (double *)calloc((size_t)N, sizeof(double));
  if (!sp || !nl || !cdf) { free(sp); free(nl); free(cdf); return ORC_E_NOMEM; }
  long long near = 0;
  double o[2] = {obs[0], m->kind == ORC_NAV2D ? obs[1] : 0.0};

  /* propagate every particle through T, reweight by Z(o | s', a) */
  for (int i = 0; i < N; ++i) {
    pstate in = {x ? x[i] : 0.0, y ? y[i] : 0.0, s ? s[i] : 0};
    if (pf) for (int q = 0; q < CR_N; ++q) { in.px[q] = pf[(2 * q) * N + i]; in.py[q] = pf[(2 * q + 1) * N + i]; }
    uint32_t w[4] = {0, 0, 0, 0};
    if (m->kind == ORC_NAV2D) draw(seed, (uint32_t)(i / 2), 3, 0, 0, 0, t_step, w);
    double r;
    const orc_ctr c = {seed, (uint32_t)i, 3, 0, 0, 0, t_step};
    model_step(m, &in, action, (i & 1) ? w[2] : w[0], (i & 1) ? w[3] : w[1], &c, &sp[i], &r, &near);
    nl[i] = lw[i] + model_loglik(m, &sp[i], action, o);
  }
  double ls = log_sum_exp(nl, N);
  if (ls == -INFINITY) { free(sp); free(nl); free(cdf); return ORC_E_DEGENERATE; }
  double sw2 = 0.0;
  for (int i = 0; i < N; ++i) { nl[i] -= ls; double w = exp(nl[i]); sw2 += w * w; }
  res->ess = 1.0 / sw2;
  res->resampled = res->ess < 0.5 * N;
  res->ess_tie = fabs(res->ess - 0.5 * N) < 1e-4 * N;
  if (res->ess_tie) ++near;
  for (int i = 0; i < N; ++i) {
    if (res->prop_x) res->prop_x[i] = sp[i].x;
    if (res->prop_y) res->prop_y[i] = sp[i].y;
    if (res->prop_s) res->prop_s[i] = sp[i].s;
    if (res->ties) res->ties[i] = 0;
  }

  if (res->resampled) {
    /* systematic resampling: positions (u0 + i)/N of the total mass, interval search */
    uint32_t w[4];
    draw(seed, 0, 4, 0, 0, 0, t_step, w);
    double u0 = orc_uniform(w[0]);
    double acc = 0.0;
    for (int k = 0; k < N; ++k) { acc += exp(nl[k]); cdf[k] = acc; }
    int k = 0;
    for (int i = 0; i < N; ++i) {
      double pos = (u0 + i) / N * cdf[N - 1];
      while (k < N - 1 && !(pos < cdf[k])) ++k;
      ancestors[i] = k;
      if (fabs(pos - cdf[k]) < 1e-5 || (k > 0 && fabs(pos - cdf[k - 1]) < 1e-5)) {
        ++near;
        if (res->ties) res->ties[i] = 1;
      }
    }
    for (int i = 0; i < N; ++i) {
      pstate a = sp[ancestors[i]];
      if (x) x[i] = a.x;
      if (y) y[i] = a.y;
      if (s) s[i] = a.s;
      if (pf) for (int q = 0; q < CR_N; ++q) { pf[(2 * q) * N + i] = a.px[q]; pf[(2 * q + 1) * N + i] = a.py[q]; }
      lw[i] = -log((double)N);
    }
  } else {
    for (int i = 0; i < N; ++i) {
      if (x) x[i] = sp[i].x;
      if (y) y[i] = sp[i].y;
      if (s) s[i] = sp[i].s;
      if (pf) for (int q = 0; q < CR_N; ++q) { pf[(2 * q) * N + i] = sp[i].px[q]; pf[(2 * q + 1) * N + i] = sp[i].py[q]; }
      lw[i] = nl[i];
      if (ancestors) ancestors[i] = i;
    }
  }
  res->near_ties = near;
  free(sp); free(nl); free(cdf);
  return ORC_OK;
}

/* Exposed pieces for the oracle's own pins. */
double orc_crowd_loglik(int32_t flags, int o) {
  pstate sp;
  memset(&sp, 0, sizeof sp);
  sp.s = flags;
  return crowd_loglik(&sp, o);
}

double orc_crowd_heuristic(double y, int32_t flags, double gamma) {
  orc_model m;
  memset(&m, 0, sizeof m);
  m.kind = ORC_CROWD;
  pstate s;
  memset(&s, 0, sizeof s);
  s.y = y;
  s.s = flags;
  return model_heuristic(&m, &s, gamma);
}

double orc_nav_heuristic(double x, double y, double gamma) {
  orc_model m;
  memset(&m, 0, sizeof m);
  pstate s = {x, y, 0};
  return model_heuristic(&m, &s, gamma);
}

int orc_grid_step(const orc_model *m, int32_t s, int a, int32_t *out, double *reward) {
  pstate in = {0.0, 0.0, s}, o;
  long long near = 0;
  model_step(m, &in, a, 0, 0, NULL, &o, reward, &near);
  *out = o.s;
  return ORC_OK;
}

double orc_grid_loglik(const orc_model *m, int32_t s, int a, int obs) {
  pstate sp = {0.0, 0.0, s};
  double o[2] = {(double)obs, 0.0};
  return model_loglik(m, &sp, a, o);
}

int orc_grid_draw_obs(const orc_model *m, int32_t s, int a, uint32_t w0) {
  pstate sp = {0.0, 0.0, s};
  double o[2];
  model_draw_obs(m, &sp, a, w0, 0, NULL, o);
  return (int)o[0];
}

void orc_nav_step(double x, double y, int a, uint32_t wa, uint32_t wb, double *ox, double *oy,
                  double *reward) {
  orc_model m;
  memset(&m, 0, sizeof m);
  pstate in = {x, y, 0}, o;
  long long near = 0;
  model_step(&m, &in, a, wa, wb, NULL, &o, reward, &near);
  *ox = o.x;
  *oy = o.y;
}

double orc_nav_loglik(double sx, double sy, double ox, double oy) {
  orc_model m;
  memset(&m, 0, sizeof m);
  pstate sp = {sx, sy, 0};
  double o[2] = {ox, oy};
  return model_loglik(&m, &sp, 0, o);
}

/* ------------------------------------------------------------------------------------ */
/* Episode mode (Alg. 1-3 as printed): every planning iteration k = 1, 2, ... samples M     */
/* episodes from the root belief and runs them to depth D_max = k, each step sampling an   */
/* action from softmax(Psi(b,.)/eta), simulating G, adding the reward and a visit to the  */
/* action node and moving to the child belief of the observation (created on first visit; */
/* continuous observations always create one); episodes that reach a terminal state stop */
/* (FilterTerminals).  The backup (Alg. 3) then aggregates the leaves' heuristics and,     */
/* for d = D_max..1, forms Q of every action node at depth d-1 from its mean reward and   */
/* the visit-weighted values of its children (normalised by the action's own visits) and  */
/* applies V_curr = L Psi, Psi <- Psi - V_curr + Q, V = L Psi to every belief at d-1.     */
/* Actions without a visit enter the update with Q = 0 (the dense tensor's default).      */
/* Node ids are assigned in creation order: iteration, depth step, episode.               */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  /* inputs */
  int M, K, O;             /* episodes per iteration, iterations (= max depth), |O| (0: continuous) */
  double eta, gamma;
  uint64_t seed;
  int cap;                 /* belief-node capacity of the arrays below                    */
  const double *root_pf;   /* CROWD root people coordinates [12][Np], or NULL             */
  /* tree arrays, capacity cap (per action node: [cap * A]; child table: [cap * A * O]) */
  int32_t *parent_an;      /* parent action node b * A + a (-1 at the root)                */
  int32_t *depth;
  double *psi, *V, *C, *Ws, *Hs;
  int64_t *N, *Nl;
  int32_t *child;
  /* results */
  int n_nodes, action;
  double v_root;
  double q_root[ORC_MAXA], policy[ORC_MAXA];
  long long particle_steps, near_decisions, near_threshold;
} orc_episode_args;

/* index of the first cumulative entry above u; flags u within tol of a boundary */
static int sample_cdf(const double *cdf, int n, double u, double tol, long long *near) {
  int i = 0;
  while (i < n - 1 && !(u < cdf[i])) ++i;
  if (fabs(u - cdf[i]) < tol || (i > 0 && fabs(u - cdf[i - 1]) < tol)) ++*near;
  return i;
}

static void ep_new_node(orc_episode_args *io, int A, int id, int parent_an, int d,
                        const double *lpi) {
  io->parent_an[id] = parent_an;
  io->depth[id] = d;
  io->V[id] = 0.0;
  io->Hs[id] = 0.0;
  io->Nl[id] = 0;
  for (int a = 0; a < A; ++a) {
    io->psi[(long long)id * A + a] = io->eta * lpi[a];
    io->C[(long long)id * A + a] = 0.0;
    io->N[(long long)id * A + a] = 0;
    for (int o = 0; o < io->O; ++o) io->child[((long long)id * A + a) * io->O + o] = -1;
  }
}

int orc_plan_episodes(const orc_model *m, const double *root_x, const double *root_y,
                      const int32_t *root_s, const double *root_w, int Np,
                      orc_episode_args *io) {
  const int A = orc_num_actions(m->kind), M = io->M, K = io->K;
  if (Np < 1 || M < 1 || K < 1 || K > ORC_MAXD || !(io->eta > 0.0) || !(io->gamma > 0.0) ||
      !(io->gamma < 1.0) || m->pi_mode == ORC_PI_NAV_DIST || io->cap < 1)
    return ORC_E_INVALID;
  if ((m->kind == ORC_NAV2D) != (io->O == 0)) return ORC_E_INVALID;
  double lpi[ORC_MAXA];
  log_pibar(m, NULL, NULL, 0, lpi);
  pstate *root = (pstate *)calloc((size_t)Np, sizeof(pstate));
  double *cdf = (double *)calloc((size_t)Np, sizeof(double));
  pstate *S = (pstate *)calloc((size_t)M, sizeof(pstate));
  int *B = (int *)calloc((size_t)M, sizeof(int)), *alive = (int *)calloc((size_t)M, sizeof(int));
  int rc = (root && cdf && S && B && alive) ? ORC_OK : ORC_E_NOMEM;
  io->n_nodes = 0;
  io->particle_steps = io->near_decisions = io->near_threshold = 0;
  io->action = -1;
  io->v_root = NAN;
  if (rc == ORC_OK) {
    /* root belief: normalised weights, terminal particles weight 0 (as the full-width plan) */
    double tot = 0.0;
    for (int i = 0; i < Np; ++i) {
      root[i].x = root_x ? root_x[i] : 0.0;
      root[i].y = root_y ? root_y[i] : 0.0;
      root[i].s = root_s ? root_s[i] : 0;
      if (io->root_pf)
        for (int q = 0; q < CR_N; ++q) {
          root[i].px[q] = io->root_pf[(2 * q) * Np + i];
          root[i].py[q] = io->root_pf[(2 * q + 1) * Np + i];
        }
      double w = root_w ? root_w[i] : 1.0;
      if (w < 0.0) rc = ORC_E_INVALID;
      if (model_is_terminal(m, &root[i])) w = 0.0;
      cdf[i] = w;
      tot += w;
    }
    if (rc == ORC_OK && !(tot > 0.0)) rc = ORC_E_DEGENERATE;
    double acc = 0.0;
    for (int i = 0; i < Np && rc == ORC_OK; ++i) { acc += cdf[i] / tot; cdf[i] = acc; }
  }
  if (rc == ORC_OK) {
    ep_new_node(io, A, 0, -1, 0, lpi);
    io->n_nodes = 1;
  }
  for (int k = 1; k <= K && rc == ORC_OK; ++k) {
    /* SampleStatesFromBelief */
    for (int e = 0; e < M; ++e) {
      uint32_t w[4];
      draw(io->seed, (uint32_t)e, 7, 0, 0, 0, (uint64_t)k, w);
      int i = sample_cdf(cdf, Np, orc_uniform(w[0]), 1e-12, &io->near_decisions);
      S[e] = root[i];
      B[e] = 0;
      alive[e] = 1;
    }
    /* Search (Alg. 2) */
    for (int d = 0; d < k && rc == ORC_OK; ++d) {
      for (int e = 0; e < M && rc == ORC_OK; ++e) {
        if (!alive[e]) continue;
        const int b = B[e];
        double z[ORC_MAXA], pc[ORC_MAXA], mx = -INFINITY, sum = 0.0;
        for (int a = 0; a < A; ++a) {
          z[a] = io->psi[(long long)b * A + a] / io->eta;
          if (z[a] > mx) mx = z[a];
        }
        for (int a = 0; a < A; ++a) { pc[a] = exp(z[a] - mx); sum += pc[a]; }
        double run = 0.0;
        for (int a = 0; a < A; ++a) { run += pc[a] / sum; pc[a] = run; }
        uint32_t w[4];
        draw(io->seed, (uint32_t)e, 8, (uint32_t)d, 0, 0, (uint64_t)k, w);
        const int a = sample_cdf(pc, A, orc_uniform(w[0]), 1e-5, &io->near_decisions);
        pstate sp;
        double r, o[2];
        draw(io->seed, (uint32_t)e, 9, (uint32_t)d, 0, 0, (uint64_t)k, w);
        const orc_ctr cs = {io->seed, (uint32_t)e, 9, (uint32_t)d, 0, 0, (uint64_t)k};
        model_step(m, &S[e], a, w[0], w[1], &cs, &sp, &r, &io->near_threshold);
        draw(io->seed, (uint32_t)e, 10, (uint32_t)d, 0, 0, (uint64_t)k, w);
        const orc_ctr co = {io->seed, (uint32_t)e, 10, (uint32_t)d, 0, 0, (uint64_t)k};
        model_draw_obs(m, &sp, a, w[0], w[1], &co, o);
        const long long an = (long long)b * A + a;
        io->C[an] += r;
        io->N[an] += 1;
        io->particle_steps += 1;
        if (model_is_terminal(m, &sp)) { alive[e] = 0; continue; }   /* FilterTerminals */
        int nb;
        if (io->O > 0) {
          const long long slot = an * io->O + (long long)o[0];
          nb = io->child[slot];
          if (nb < 0) {
            if (io->n_nodes >= io->cap) { rc = ORC_E_NOMEM; break; }
            nb = io->n_nodes++;
            ep_new_node(io, A, nb, (int)an, d + 1, lpi);
            io->child[slot] = nb;
          }
        } else {
          if (io->n_nodes >= io->cap) { rc = ORC_E_NOMEM; break; }
          nb = io->n_nodes++;
          ep_new_node(io, A, nb, (int)an, d + 1, lpi);
        }
        B[e] = nb;
        S[e] = sp;
      }
    }
    if (rc != ORC_OK) break;
    /* leaves: ValueHeuristic aggregated per leaf belief */
    for (int e = 0; e < M; ++e) {
      if (!alive[e]) continue;
      io->Hs[B[e]] += model_heuristic(m, &S[e], io->gamma);
      io->Nl[B[e]] += 1;
    }
    /* Backup (Alg. 3) */
    for (int n = 0; n < io->n_nodes; ++n)
      if (io->depth[n] == k) io->V[n] = io->Nl[n] > 0 ? io->Hs[n] / (double)io->Nl[n] : 0.0;
    for (int d = k; d >= 1; --d) {
      for (long long x = 0; x < (long long)io->n_nodes * A; ++x) io->Ws[x] = 0.0;
      for (int n = 0; n < io->n_nodes; ++n) {
        if (io->depth[n] != d) continue;
        double visits = 0.0;
        if (d == k) visits = (double)io->Nl[n];
        else for (int a = 0; a < A; ++a) visits += (double)io->N[(long long)n * A + a];
        io->Ws[io->parent_an[n]] += visits * io->V[n];
      }
      for (int n = 0; n < io->n_nodes; ++n) {
        if (io->depth[n] != d - 1) continue;
        double q[ORC_MAXA], *ps = io->psi + (long long)n * A;
        for (int a = 0; a < A; ++a) {
          const long long an = (long long)n * A + a;
          q[a] = io->N[an] > 0 ? io->C[an] / (double)io->N[an] +
                                     io->gamma * io->Ws[an] / (double)io->N[an]
                               : 0.0;
        }
        const double vcur = lse_value(ps, A, io->eta);
        for (int a = 0; a < A; ++a) ps[a] = ps[a] - vcur + q[a];
        io->V[n] = lse_value(ps, A, io->eta);
        if (n == 0)
          for (int a = 0; a < A; ++a) io->q_root[a] = q[a];
      }
    }
  }
  if (rc == ORC_OK) {
    const double *ps = io->psi;
    int best = 0;
    for (int a = 0; a < A; ++a) if (ps[a] > ps[best]) best = a;
    io->action = best;
    io->v_root = io->V[0];
    for (int a = 0; a < A; ++a) io->policy[a] = exp((ps[a] - io->V[0]) / io->eta);
  }
  free(root); free(cdf); free(S); free(B); free(alive);
  return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Environment of the closed loop (Alg. 1: execute the action, perceive the observation):  */
/* the true state steps under the model's own transition and observation processes, with   */
/* its own random numbers (purposes 5 and 6, node = time step t).                          */
/* ------------------------------------------------------------------------------------ */
int orc_env_step(const orc_model *m, double *x, double *y, int32_t *s, double *pf, int a,
                 uint64_t seed, uint64_t t, double obs[2], double *reward, int *terminal) {
  if (a < 0 || a >= orc_num_actions(m->kind)) return ORC_E_INVALID;
  pstate in = {*x, *y, *s}, out;
  if (pf) for (int q = 0; q < CR_N; ++q) { in.px[q] = pf[2 * q]; in.py[q] = pf[2 * q + 1]; }
  long long near = 0;
  uint32_t w[4];
  draw(seed, 0, 5, 0, 0, 0, t, w);
  const orc_ctr cs = {seed, 0, 5, 0, 0, 0, t}, co = {seed, 0, 6, 0, 0, 0, t};
  model_step(m, &in, a, w[0], w[1], &cs, &out, reward, &near);
  draw(seed, 0, 6, 0, 0, 0, t, w);
  model_draw_obs(m, &out, a, w[0], w[1], &co, obs);
  if (pf) for (int q = 0; q < CR_N; ++q) { pf[2 * q] = out.px[q]; pf[2 * q + 1] = out.py[q]; }
  *terminal = model_is_terminal(m, &out);
  *x = out.x;
  *y = out.y;
  *s = out.s;
  return ORC_OK;
}

double orc_belief_value(const double *q, const double *lpi, int A, double eta) {
  return belief_value(q, lpi, A, eta);
}
