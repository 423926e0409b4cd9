/*
 * bcts_oracle.c -- the ORACLE: plain, slow, obviously correct CPU reference of
 * the Batch-BFS / BCTS search, in FP64.  TEST INFRASTRUCTURE ONLY: the tests,
 * the smoke check and the bench's CPU-baseline leg call it; the product path
 * never does.  It shares no code, header, table or constant with the CUDA
 * library: every constant below is written here from the environment
 * definition, independently.
 *
 * What it computes (paper: "Improve Agents without Retraining: Parallel Tree
 * Search with Off-Policy Correction", Hallak et al., NeurIPS 2021):
 *   - Eq. 1: the d-step Q estimate, max over a_1..a_d of the discounted d-step
 *     return plus gamma^d Q(s_d, a_d), computed by a recursive depth-first search
 *     (the max over the tail factorises level by level);
 *   - Prop. 1 / Sec. 3.3: the Bellman errors delta(a) = Q_1(s,a) - Q_0(s,a) from
 *     the root and the depth-1 nodes;
 *   - Eq. 7: the Bellman penalty B(delta_e, delta_o, A, d), or (exact mode) the
 *     bias gap B_e - B_o of Lemma 2 itself, with sigma = delta / sqrt(2);
 *   - Eq. 3 / Eq. 4: the corrected values and the BCTS action.
 * The environment is the synthetic sprite environment that stands in for the
 * paper's Atari games (Sec. 4 uses CuLE); the Q-network is Nature-DQN with
 * seeded weights standing in for the pre-trained Rainbow agent (Sec. 5.1),
 * fed the 4-frame stack of Sec. 5 (frame stacking).
 *
 * Readings of the paper taken here (each listed with its reason in the design
 * notes): |delta| as the std-dev surrogate; delta_e = arithmetic mean of
 * |delta(a)| over a != pi_o; natural log in Eq. 7; Eq. 7 applied unchanged for
 * every d >= 1 (sqrt(d-1) = 0 at d = 1); d = 0 returns pi_o; ties broken to the
 * lowest index; the correction is scaled by the swept multiplier c (Sec. 5.1).
 *
 * Pins: tests/test_oracle_*.py check this file against brute-force enumeration
 * of all A^d action sequences, torch.nn.functional conv2d/linear in float64,
 * closed-form returns of hand-built environments, the Lemma 3 form of Eq. 7
 * and the exact GEV biases of Lemma 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- state: 80 bytes, same field order and sizes as the documented layout -- */
typedef struct {
    int16_t pos[4][4][2]; /* [history slot][object][x,y]; slot 3 newest */
    int8_t vel[4][2];     /* object velocities; object 0 = agent, unused */
    uint32_t tick;
    uint32_t pad;
} or_state;

enum { OR_GRID = 21, OR_HIST = 4, OR_NOBJ = 4, OR_PIX = 84 };

/* ---- environment step ---------------------------------------------------- */
/* Agent move table: action a, direction a mod 9, speed 1 + a / 9. */
static const int OR_DX[9] = {0, 0, 1, -1, 0, 1, -1, 1, -1};
static const int OR_DY[9] = {0, -1, 0, 0, 1, -1, -1, 1, 1};

static int or_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* lowbias32 integer hash (C. Wellons, "hash prospector", 2018). */
static uint32_t or_hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

/* Reflect one coordinate moving by v off the walls at 0 and GRID-1. */
static void or_reflect(int *p, int *v) {
    int q = *p + *v;
    if (q < 0) { q = -q; *v = -*v; }
    if (q > OR_GRID - 1) { q = 2 * (OR_GRID - 1) - q; *v = -*v; }
    *p = q;
}

/* One tick of the deterministic sprite environment (the forward model G of
 * Alg. 1).  Returns the integer reward in {-1, 0, 1}. */
int or_env_step(const or_state *s, int a, or_state *out) {
    or_state n = *s;
    int ax = s->pos[3][0][0], ay = s->pos[3][0][1];
    int dir = a % 9, speed = 1 + a / 9;
    int nax = or_clampi(ax + speed * OR_DX[dir], 0, OR_GRID - 1);
    int nay = or_clampi(ay + speed * OR_DY[dir], 0, OR_GRID - 1);
    int px[4], py[4];
    px[0] = nax;
    py[0] = nay;
    for (int k = 1; k < OR_NOBJ; ++k) {
        int x = s->pos[3][k][0], y = s->pos[3][k][1];
        int vx = s->vel[k][0], vy = s->vel[k][1];
        or_reflect(&x, &vx);
        or_reflect(&y, &vy);
        px[k] = x;
        py[k] = y;
        n.vel[k][0] = (int8_t)vx;
        n.vel[k][1] = (int8_t)vy;
    }
    int reward = 0;
    for (int k = 1; k < OR_NOBJ; ++k) {
        if (px[k] == nax && py[k] == nay) {
            reward += (k == 1) ? 1 : -1;
            uint32_t key = s->tick * 0x9E3779B1u + (uint32_t)k * 0x85EBCA77u +
                           (uint32_t)(nax * OR_GRID + nay) * 0xC2B2AE3Du;
            uint32_t h = or_hash32(key);
            px[k] = (int)(h % OR_GRID);
            py[k] = (int)((h >> 16) % OR_GRID);
        }
    }
    if (reward > 1) reward = 1;
    if (reward < -1) reward = -1;
    for (int h = 0; h < OR_HIST - 1; ++h) memcpy(n.pos[h], s->pos[h + 1], sizeof n.pos[h]);
    for (int k = 0; k < OR_NOBJ; ++k) {
        n.pos[3][k][0] = (int16_t)px[k];
        n.pos[3][k][1] = (int16_t)py[k];
    }
    n.tick = s->tick + 1u;
    n.pad = 0;
    *out = n;
    return reward;
}

/* ---- renderer: 4 x 84 x 84 uint8 frame stack, channel h = history slot h ---- */
/* Sprite masks, 4x4, bit (r*4 + c) set = pixel drawn. */
static const uint16_t OR_SPRITE[4] = {0xFFFF, 0x6FF6, 0x9669, 0xF99F};
static const uint8_t OR_PALETTE[4] = {240, 192, 128, 64};

void or_render(const or_state *s, uint8_t *frames) {
    memset(frames, 0, OR_HIST * OR_PIX * OR_PIX);
    for (int h = 0; h < OR_HIST; ++h) {
        uint8_t *f = frames + h * OR_PIX * OR_PIX;
        for (int k = 0; k < OR_NOBJ; ++k) { /* later objects paint over earlier ones */
            int cx = s->pos[h][k][0], cy = s->pos[h][k][1];
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c)
                    if ((OR_SPRITE[k] >> (r * 4 + c)) & 1)
                        f[(cy * 4 + r) * OR_PIX + (cx * 4 + c)] = OR_PALETTE[k];
        }
    }
}

/* ---- Nature-DQN forward in FP64 with direct loops ------------------------- */
/* Weights: flat float32 in PyTorch parameter order (conv [Cout][Cin][kh][kw],
 * bias; linear [out][in], bias; fc1 input flattened (C, H, W)).  Input pixels
 * are scaled by 1/255. */
static void or_conv_relu(const double *in, int cin, int ih, int iw, const float *w, const float *b,
                         int cout, int k, int stride, double *out, int oh, int ow) {
    for (int o = 0; o < cout; ++o)
        for (int y = 0; y < oh; ++y)
            for (int x = 0; x < ow; ++x) {
                double acc = (double)b[o];
                for (int c = 0; c < cin; ++c)
                    for (int ky = 0; ky < k; ++ky)
                        for (int kx = 0; kx < k; ++kx)
                            acc += (double)w[((o * cin + c) * k + ky) * k + kx] *
                                   in[(c * ih + (y * stride + ky)) * iw + (x * stride + kx)];
                out[(o * oh + y) * ow + x] = acc > 0.0 ? acc : 0.0;
            }
}

static void or_linear(const double *in, int nin, const float *w, const float *b, int nout, int relu,
                      double *out) {
    for (int o = 0; o < nout; ++o) {
        double acc = (double)b[o];
        for (int i = 0; i < nin; ++i) acc += (double)w[(size_t)o * nin + i] * in[i];
        out[o] = (relu && acc < 0.0) ? 0.0 : acc;
    }
}

size_t or_qnet_numel(int A) {
    return (size_t)32 * 4 * 8 * 8 + 32 + 64 * 32 * 4 * 4 + 64 + 64 * 64 * 3 * 3 + 64 +
           (size_t)512 * 3136 + 512 + (size_t)A * 512 + A;
}

void or_qnet(const uint8_t *frames, const float *W, int A, double *q) {
    const float *c1w = W, *c1b = c1w + 32 * 4 * 8 * 8;
    const float *c2w = c1b + 32, *c2b = c2w + 64 * 32 * 4 * 4;
    const float *c3w = c2b + 64, *c3b = c3w + 64 * 64 * 3 * 3;
    const float *f1w = c3b + 64, *f1b = f1w + (size_t)512 * 3136;
    const float *f2w = f1b + 512, *f2b = f2w + (size_t)A * 512;
    double *x = malloc(sizeof(double) * 4 * 84 * 84);
    double *h1 = malloc(sizeof(double) * 32 * 20 * 20);
    double *h2 = malloc(sizeof(double) * 64 * 9 * 9);
    double *h3 = malloc(sizeof(double) * 64 * 7 * 7);
    double *h4 = malloc(sizeof(double) * 512);
    for (int i = 0; i < 4 * 84 * 84; ++i) x[i] = (double)frames[i] / 255.0;
    or_conv_relu(x, 4, 84, 84, c1w, c1b, 32, 8, 4, h1, 20, 20);
    or_conv_relu(h1, 32, 20, 20, c2w, c2b, 64, 4, 2, h2, 9, 9);
    or_conv_relu(h2, 64, 9, 9, c3w, c3b, 64, 3, 1, h3, 7, 7);
    or_linear(h3, 3136, f1w, f1b, 512, 1, h4);
    or_linear(h4, 512, f2w, f2b, A, 0, q);
    free(x); free(h1); free(h2); free(h3); free(h4);
}

/* Q-values of a state: render the stack, run the network. */
static void or_q_of_state(const or_state *s, const float *W, int A, double *q) {
    uint8_t fr[4 * 84 * 84];
    or_render(s, fr);
    or_qnet(fr, W, A, q);
}

/* Batch of frame stacks -> Q [n][A], parallel over stacks. */
void or_qnet_batch(const uint8_t *frames, int n, const float *W, int A, double *q) {
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < n; ++i) or_qnet(frames + (size_t)i * 4 * 84 * 84, W, A, q + (size_t)i * A);
}

static int or_argmax_lowest(const double *v, int n) {
    int best = 0;
    for (int i = 1; i < n; ++i)
        if (v[i] > v[best]) best = i;
    return best;
}

static double or_maxv(const double *v, int n) { return v[or_argmax_lowest(v, n)]; }

/* W_k(s): value of a node at depth k <= d.  At k = d it is max_a Q(s, a)
 * (Alg. 1's leaf term); above, max over actions of r + gamma * W_{k+1}(s'),
 * which equals the max over the remaining action sequence in Eq. 1. */
static double or_node_value(const or_state *s, int k, int d, const float *W, int A, double gamma) {
    if (k == d) {
        double q[64];
        or_q_of_state(s, W, A, q);
        return or_maxv(q, A);
    }
    double best = -INFINITY;
    for (int a = 0; a < A; ++a) {
        or_state n;
        int r = or_env_step(s, a, &n);
        double v = (double)r + gamma * or_node_value(&n, k + 1, d, W, A, gamma);
        if (v > best) best = v;
    }
    return best;
}

/* Eq. 7: B = sqrt(log A) (de sqrt(d) - do sqrt(d-1)) - (de - do) / sqrt(8). */
double or_bellman_penalty(double delta_e, double delta_o, int A, int d) {
    double dm1 = d >= 1 ? (double)(d - 1) : 0.0;
    return sqrt(log((double)A)) * (delta_e * sqrt((double)d) - delta_o * sqrt(dm1)) -
           (delta_e - delta_o) / sqrt(8.0);
}

/*
 * Normal upper-tail quantile: the x with Q(x) = 1 - Phi(x) = q, 0 < q < 1, by
 * bisection on Q(x) = erfc(x / sqrt 2) / 2 (monotone decreasing) until the
 * bracket stops shrinking in double precision.  Phi^-1(1 - q) = this x.
 */
double or_normal_upper_quantile(double q) {
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (0.5 * erfc(mid / sqrt(2.0)) > q)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/*
 * Lemma 2: the expected shift of the maximum of m iid standard normals as its
 * GEV mean, Phi^-1(1 - 1/m) + gamma_EM * sigma_GEV with
 * sigma_GEV = Phi^-1(1 - 1/(e m)) - Phi^-1(1 - 1/m) (the Lemma 1 parameters);
 * 0 for a single element (m <= 1), as the lemma states for its d = 1 cases.
 */
static double or_gev_shift(double m) {
    const double euler_gamma = 0.57721566490153286061;
    if (m <= 1.0) return 0.0;
    double x1 = or_normal_upper_quantile(1.0 / m);
    double xe = or_normal_upper_quantile(1.0 / (exp(1.0) * m));
    return x1 + euler_gamma * (xe - x1);
}

/*
 * Exact bias gap of Eq. 3: B_e(sigma_e, A, d) - B_o(sigma_o, A, d) of Lemma 2,
 * the maximum over A^d - A^(d-1) leaves (a_0 != pi_o) against A^(d-1) leaves
 * (a_0 = pi_o), with the standard deviations estimated as delta / sqrt(2)
 * (Prop. 1).
 */
double or_bellman_penalty_exact(double delta_e, double delta_o, int A, int d) {
    double n_o = pow((double)A, (double)(d - 1));
    double n_e = pow((double)A, (double)d) - n_o;
    return delta_e / sqrt(2.0) * or_gev_shift(n_e) - delta_o / sqrt(2.0) * or_gev_shift(n_o);
}

/*
 * Full search from one root.
 *   values[A]  : corrected root values Q^BCTS_d(s0, a) (Eq. 3); for d = 0, Q_0(s0, a)
 *   *action    : lowest-index argmax of values (Eq. 4)
 *   exact_gev: 0 = Eq. 7's penalty, 1 = Lemma 2's exact bias gap
 *   diag (may be NULL), 4*A + 4 doubles:
 *     [0,A)    Q_0(s0, a)                      root Q-values
 *     [A,2A)   V_d(s0, a)                      uncorrected Eq. 1 values
 *     [2A,3A)  delta(a) = r(s0,a) + gamma max Q(s1^a) - Q_0(s0,a)   (Prop. 1)
 *     [3A,4A)  r(s0, a)
 *     4A: pi_o, 4A+1: delta_o, 4A+2: delta_e, 4A+3: B (Eq. 7)
 * Work is split over the A root actions (OpenMP) when `parallel` is set.
 */
static void or_search_one(const or_state *root, const float *W, int A, int d, double gamma, double corr,
                          int exact_gev, int parallel, int *action, double *values, double *diag) {
    double q0[64], V[64], delta[64], r0[64];
    or_q_of_state(root, W, A, q0);
    int pi_o = or_argmax_lowest(q0, A);
    if (d == 0) {
        for (int a = 0; a < A; ++a) values[a] = q0[a];
        *action = pi_o;
        if (diag) {
            for (int a = 0; a < A; ++a) {
                diag[a] = q0[a]; diag[A + a] = q0[a]; diag[2 * A + a] = 0.0; diag[3 * A + a] = 0.0;
            }
            diag[4 * A] = pi_o; diag[4 * A + 1] = 0; diag[4 * A + 2] = 0; diag[4 * A + 3] = 0;
        }
        return;
    }
#pragma omp parallel for schedule(dynamic) if (parallel)
    for (int a = 0; a < A; ++a) {
        or_state s1;
        int r = or_env_step(root, a, &s1);
        double q1[64];
        or_q_of_state(&s1, W, A, q1);
        double maxq1 = or_maxv(q1, A);
        r0[a] = (double)r;
        delta[a] = (double)r + gamma * maxq1 - q0[a];
        double tail = (d == 1) ? maxq1 : or_node_value(&s1, 1, d, W, A, gamma);
        V[a] = (double)r + gamma * tail;
    }
    double delta_o = fabs(delta[pi_o]);
    double delta_e = 0.0;
    if (A > 1) {
        for (int a = 0; a < A; ++a)
            if (a != pi_o) delta_e += fabs(delta[a]);
        delta_e /= (double)(A - 1);
    }
    double B = exact_gev ? or_bellman_penalty_exact(delta_e, delta_o, A, d)
                         : or_bellman_penalty(delta_e, delta_o, A, d);
    double gd = pow(gamma, (double)d);
    for (int a = 0; a < A; ++a) values[a] = (a == pi_o) ? V[a] : V[a] - gd * corr * B;
    *action = or_argmax_lowest(values, A);
    if (diag) {
        for (int a = 0; a < A; ++a) {
            diag[a] = q0[a]; diag[A + a] = V[a]; diag[2 * A + a] = delta[a]; diag[3 * A + a] = r0[a];
        }
        diag[4 * A] = pi_o; diag[4 * A + 1] = delta_o; diag[4 * A + 2] = delta_e; diag[4 * A + 3] = B;
    }
}

/* n roots; roots run one after another, each root's A subtrees in parallel. */
int or_search_ex(const or_state *roots, int n, const float *W, int A, int d, double gamma, double corr,
                 int exact_gev, int *actions, double *values, double *diag) {
    if (A < 1 || A > 64 || d < 0 || n < 0) return -1;
    for (int i = 0; i < n; ++i)
        or_search_one(&roots[i], W, A, d, gamma, corr, exact_gev, 1, &actions[i], values + (size_t)i * A,
                      diag ? diag + (size_t)i * (4 * A + 4) : NULL);
    return 0;
}

int or_search(const or_state *roots, int n, const float *W, int A, int d, double gamma, double corr,
              int *actions, double *values, double *diag) {
    return or_search_ex(roots, n, W, A, d, gamma, corr, 0, actions, values, diag);
}

/*
 * Alg. 1's backup and the BCTS correction on given leaf data, n roots:
 *   leaf_R, leaf_maxq : n * A^d leaves in Alg. 1's order (child = parent * A + a),
 *                       accumulated discounted reward R and max_a Q of each leaf
 *   q0, r1, maxq1     : n * A, root Q-values, r(s_0, a) and max_a' Q(s_1^a, a')
 * V(a_0) = max over the A^(d-1) leaves below root action a_0 of R + gamma^d maxq
 * (Eq. 1 in its flat form; Alg. 1's argmax over the leaves), delta(a) = r1 +
 * gamma maxq1 - q0 (Prop. 1), the penalty (Eq. 7, or Lemma 2's gap when
 * exact_gev), values (Eq. 3) and the action (Eq. 4).  d = 0 returns q0 and pi_o.
 */
int or_backup(const double *leaf_R, const double *leaf_maxq, const double *q0, const double *r1,
              const double *maxq1, int n, int A, int d, double gamma, double corr, int exact_gev, int *actions,
              double *values) {
    if (A < 1 || A > 64 || d < 0 || n < 0) return -1;
    long long seg = 1;
    for (int i = 1; i < d; ++i) seg *= A;
    double gd = pow(gamma, (double)d);
    for (int i = 0; i < n; ++i) {
        const double *q = q0 + (size_t)i * A;
        double *val = values + (size_t)i * A;
        int pi_o = or_argmax_lowest(q, A);
        if (d == 0) {
            for (int a = 0; a < A; ++a) val[a] = q[a];
            actions[i] = pi_o;
            continue;
        }
        double V[64], delta[64];
        for (int a = 0; a < A; ++a) {
            long long first = ((long long)i * A + a) * seg;
            double best = -INFINITY;
            for (long long j = 0; j < seg; ++j) {
                double v = leaf_R[first + j] + gd * leaf_maxq[first + j];
                if (v > best) best = v;
            }
            V[a] = best;
            delta[a] = r1[(size_t)i * A + a] + gamma * maxq1[(size_t)i * A + a] - q[a];
        }
        double delta_o = fabs(delta[pi_o]), delta_e = 0.0;
        if (A > 1) {
            for (int a = 0; a < A; ++a)
                if (a != pi_o) delta_e += fabs(delta[a]);
            delta_e /= (double)(A - 1);
        }
        double B = exact_gev ? or_bellman_penalty_exact(delta_e, delta_o, A, d)
                             : or_bellman_penalty(delta_e, delta_o, A, d);
        for (int a = 0; a < A; ++a) val[a] = (a == pi_o) ? V[a] : V[a] - gd * corr * B;
        actions[i] = or_argmax_lowest(val, A);
    }
    return 0;
}

/* ---- tree enumeration in Alg. 1 order ------------------------------------ */
/* Replay node `idx` of level `depth` (0 <= idx < A^depth): its actions are the
 * base-A digits of idx, most significant first (child = parent * A + a).
 * Returns the state and R = sum_t gamma^t r_t (Alg. 1's accumulated reward). */
void or_replay(const or_state *root, int A, int depth, long long idx, double gamma, or_state *out,
               double *R);

/*
 * One node of the tree export (Sec. 4: Batch-BFS exposes every node's cumulative
 * reward and estimated value): node idx of depth `level` (Alg. 1 order) of the
 * search from `root` to depth d.  *R = the discounted reward accumulated from the
 * root (Alg. 1's R); *V = the node's (d - level)-step value, max over the
 * remaining actions of the discounted return plus gamma^(d-level) max_a Q at the
 * leaf (the same recursion as Eq. 1's tail).
 */
void or_tree_node(const or_state *root, const float *W, int A, int d, double gamma, int level, long long idx,
                  double *R, double *V) {
    or_state s;
    or_replay(root, A, level, idx, gamma, &s, R);
    *V = or_node_value(&s, level, d, W, A, gamma);
}

void or_replay(const or_state *root, int A, int depth, long long idx, double gamma, or_state *out,
               double *R) {
    int acts[32];
    long long x = idx;
    for (int i = depth - 1; i >= 0; --i) {
        acts[i] = (int)(x % A);
        x /= A;
    }
    or_state s = *root;
    double acc = 0.0, g = 1.0;
    for (int i = 0; i < depth; ++i) {
        or_state n;
        int r = or_env_step(&s, acts[i], &n);
        acc += g * (double)r;
        g *= gamma;
        s = n;
    }
    *out = s;
    *R = acc;
}

/* Nodes [first, first+count) of level `depth` below one root. */
void or_level(const or_state *root, int A, int depth, long long first, long long count, double gamma,
              or_state *out, double *R) {
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < count; ++i) or_replay(root, A, depth, first + i, gamma, &out[i], &R[i]);
}

/* ==========================================================================
 * DNN forward-model workload (Sec. 4, runtime experiments: a randomly
 * initialised network standing in for a learned forward model; three hidden
 * layers of width 100 on a 100-wide state and a one-hot action).
 * Parameter order (PyTorch [out][in]): fm1.w [100][100+A], fm1.b, fm2.w
 * [100][100], fm2.b, fm3.w [100][100], fm3.b, fmo.w [101][100], fmo.b [101],
 * q.w [A][100], q.b [A].  Step: x = [s; onehot(a)], h_k = ReLU(W_k h_{k-1} + b_k)
 * for k = 1..3, o = W_o h_3 + b_o, s' = tanh(o[0..99]), r = o[100].  The leaf
 * value network is the linear head Q(s) = W_q s + b_q.
 * ========================================================================== */
enum { OR_DNN_D = 100, OR_DNN_H = 100 };

typedef struct {
    const float *w1, *b1, *w2, *b2, *w3, *b3, *wo, *bo, *wq, *bq;
} or_dnn_w;

static or_dnn_w or_dnn_view(const float *W, int A) {
    or_dnn_w v;
    const int D = OR_DNN_D, H = OR_DNN_H;
    v.w1 = W; v.b1 = v.w1 + (size_t)H * (D + A);
    v.w2 = v.b1 + H; v.b2 = v.w2 + (size_t)H * H;
    v.w3 = v.b2 + H; v.b3 = v.w3 + (size_t)H * H;
    v.wo = v.b3 + H; v.bo = v.wo + (size_t)(D + 1) * H;
    v.wq = v.bo + D + 1; v.bq = v.wq + (size_t)A * D;
    return v;
}

size_t or_dnn_numel(int A) {
    const size_t D = OR_DNN_D, H = OR_DNN_H;
    return H * (D + A) + H + 2 * (H * H + H) + (D + 1) * H + (D + 1) + (size_t)A * D + (size_t)A;
}

/* One forward-model step from s with action a: next state into out, returns r. */
double or_dnn_step(const double *s, int a, const float *W, int A, double *out) {
    const int D = OR_DNN_D, H = OR_DNN_H;
    or_dnn_w w = or_dnn_view(W, A);
    double h1[OR_DNN_H], h2[OR_DNN_H], h3[OR_DNN_H];
    for (int j = 0; j < H; ++j) {
        double acc = w.b1[j];
        for (int k = 0; k < D; ++k) acc += (double)w.w1[(size_t)j * (D + A) + k] * s[k];
        acc += (double)w.w1[(size_t)j * (D + A) + D + a]; /* the one-hot action input */
        h1[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int j = 0; j < H; ++j) {
        double acc = w.b2[j];
        for (int k = 0; k < H; ++k) acc += (double)w.w2[(size_t)j * H + k] * h1[k];
        h2[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int j = 0; j < H; ++j) {
        double acc = w.b3[j];
        for (int k = 0; k < H; ++k) acc += (double)w.w3[(size_t)j * H + k] * h2[k];
        h3[j] = acc > 0.0 ? acc : 0.0;
    }
    double r = 0.0;
    for (int j = 0; j <= D; ++j) {
        double acc = w.bo[j];
        for (int k = 0; k < H; ++k) acc += (double)w.wo[(size_t)j * H + k] * h3[k];
        if (j < D)
            out[j] = tanh(acc);
        else
            r = acc;
    }
    return r;
}

/* Q(s, .) = W_q s + b_q. */
void or_dnn_q(const double *s, const float *W, int A, double *q) {
    const int D = OR_DNN_D;
    or_dnn_w w = or_dnn_view(W, A);
    for (int a = 0; a < A; ++a) {
        double acc = w.bq[a];
        for (int k = 0; k < D; ++k) acc += (double)w.wq[(size_t)a * D + k] * s[k];
        q[a] = acc;
    }
}

/* Eq. 1's tail from a depth-k node, as for the sprite world. */
static double or_dnn_value(const double *s, int k, int d, const float *W, int A, double gamma) {
    double q[64];
    if (k == d) {
        or_dnn_q(s, W, A, q);
        return or_maxv(q, A);
    }
    double best = -INFINITY;
    for (int a = 0; a < A; ++a) {
        double n[OR_DNN_D];
        double r = or_dnn_step(s, a, W, A, n);
        double v = r + gamma * or_dnn_value(n, k + 1, d, W, A, gamma);
        if (v > best) best = v;
    }
    return best;
}

/*
 * BCTS search over the DNN model from n float32 roots [n][100]; outputs and
 * diag layout as or_search_ex (Eq. 1, Prop. 1, Eq. 3, Eq. 4; Eq. 7 or Lemma 2).
 */
int or_dnn_search(const float *roots, int n, const float *W, int A, int d, double gamma, double corr,
                  int exact_gev, int *actions, double *values, double *diag) {
    if (A < 1 || A > 64 || d < 0 || n < 0) return -1;
    for (int i = 0; i < n; ++i) {
        double s0[OR_DNN_D], q0[64], V[64], delta[64], r0[64];
        for (int k = 0; k < OR_DNN_D; ++k) s0[k] = (double)roots[(size_t)i * OR_DNN_D + k];
        or_dnn_q(s0, W, A, q0);
        int pi_o = or_argmax_lowest(q0, A);
        double *val = values + (size_t)i * A;
        double *dg = diag ? diag + (size_t)i * (4 * A + 4) : NULL;
        if (d == 0) {
            for (int a = 0; a < A; ++a) val[a] = q0[a];
            actions[i] = pi_o;
            if (dg) {
                for (int a = 0; a < A; ++a) { dg[a] = q0[a]; dg[A + a] = q0[a]; dg[2 * A + a] = 0; dg[3 * A + a] = 0; }
                dg[4 * A] = pi_o; dg[4 * A + 1] = 0; dg[4 * A + 2] = 0; dg[4 * A + 3] = 0;
            }
            continue;
        }
#pragma omp parallel for schedule(dynamic)
        for (int a = 0; a < A; ++a) {
            double s1[OR_DNN_D], q1[64];
            double r = or_dnn_step(s0, a, W, A, s1);
            or_dnn_q(s1, W, A, q1);
            r0[a] = r;
            delta[a] = r + gamma * or_maxv(q1, A) - q0[a];
            double tail = (d == 1) ? or_maxv(q1, A) : or_dnn_value(s1, 1, d, W, A, gamma);
            V[a] = r + gamma * tail;
        }
        double delta_o = fabs(delta[pi_o]), delta_e = 0.0;
        if (A > 1) {
            for (int a = 0; a < A; ++a)
                if (a != pi_o) delta_e += fabs(delta[a]);
            delta_e /= (double)(A - 1);
        }
        double B = exact_gev ? or_bellman_penalty_exact(delta_e, delta_o, A, d)
                             : or_bellman_penalty(delta_e, delta_o, A, d);
        double gd = pow(gamma, (double)d);
        for (int a = 0; a < A; ++a) val[a] = (a == pi_o) ? V[a] : V[a] - gd * corr * B;
        actions[i] = or_argmax_lowest(val, A);
        if (dg) {
            for (int a = 0; a < A; ++a) { dg[a] = q0[a]; dg[A + a] = V[a]; dg[2 * A + a] = delta[a]; dg[3 * A + a] = r0[a]; }
            dg[4 * A] = pi_o; dg[4 * A + 1] = delta_o; dg[4 * A + 2] = delta_e; dg[4 * A + 3] = B;
        }
    }
    return 0;
}

/* ==========================================================================
 * Pruned Batch-BFS (Sec. 4: pruning by an index array of unpruned states,
 * updated at each pruning step and used to trace the best root action).  The
 * criterion is the cumulative reward plus the estimated value the same passage
 * points to: within the subtree of each root action a_0, the nodes of every
 * level i = 2 .. d-1 are ranked by R + gamma^i max_a Q(s, a) and only the
 * `keep` best (lowest candidate index among equal scores) are expanded further;
 * a level's candidates are the children of the previous level's survivors in
 * the order survivor-index x A + a, survivors kept in increasing index order.
 * V(a_0) = max over the surviving leaves of R + gamma^d max_a Q; pi_o, the
 * Bellman errors and the penalty (Eq. 7, or Lemma 2) are the full search's.
 * diag: 4*A + 5 doubles, as or_search_ex plus [4A+4] = the smallest positive gap
 * between a kept and a dropped score over all selections of the root (+inf if
 * none; scores that are exactly equal belong to identical states and tie the
 * same way in any precision).
 * ========================================================================== */
typedef struct {
    double score;
    int idx;
} or_cand;

static int or_cand_cmp(const void *pa, const void *pb) {
    const or_cand *a = (const or_cand *)pa, *b = (const or_cand *)pb;
    if (a->score != b->score) return a->score > b->score ? -1 : 1; /* higher score first */
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);       /* then lower index */
}

static int or_int_cmp(const void *pa, const void *pb) {
    int a = *(const int *)pa, b = *(const int *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* V(a_0) of one root-action subtree under the pruning rule; *gap <- min margin. */
static double or_pruned_subtree(const or_state *s1, double R1, const float *W, int A, int d, double gamma,
                                int keep, double *gap) {
    int cnt = 1;
    or_state *lvl = (or_state *)malloc(sizeof(or_state));
    double *R = (double *)malloc(sizeof(double));
    lvl[0] = *s1;
    R[0] = R1;
    double gprev = 1.0, gp = gamma; /* gamma^(i-1), gamma^i at level i */
    for (int i = 2; i <= d; ++i) {
        gprev = gp;
        gp *= gamma;
        int nc = cnt * A;
        or_state *ch = (or_state *)malloc(sizeof(or_state) * (size_t)nc);
        double *Rc = (double *)malloc(sizeof(double) * (size_t)nc);
        double *mq = (double *)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for schedule(dynamic)
        for (int j = 0; j < nc; ++j) {
            int r = or_env_step(&lvl[j / A], j % A, &ch[j]);
            Rc[j] = R[j / A] + gprev * (double)r; /* the reward of step i-1 carries gamma^(i-1) */
            double q[64];
            or_q_of_state(&ch[j], W, A, q);
            mq[j] = or_maxv(q, A);
        }
        free(lvl);
        free(R);
        if (i == d) {
            double best = -INFINITY;
            for (int j = 0; j < nc; ++j) {
                double v = Rc[j] + gp * mq[j];
                if (v > best) best = v;
            }
            free(ch);
            free(Rc);
            free(mq);
            return best;
        }
        int k = nc < keep ? nc : keep;
        or_cand *c = (or_cand *)malloc(sizeof(or_cand) * (size_t)nc);
        for (int j = 0; j < nc; ++j) {
            c[j].score = Rc[j] + gp * mq[j];
            c[j].idx = j;
        }
        qsort(c, (size_t)nc, sizeof(or_cand), or_cand_cmp);
        if (k < nc) {
            /* the smallest positive difference between a kept and a dropped score:
             * exactly equal scores (identical states) tie in any precision and
             * are resolved by index on both sides */
            double a = c[k - 1].score, b = c[k].score;
            for (int m = k; m < nc; ++m)
                if (c[m].score < a) {
                    if (a - c[m].score < *gap) *gap = a - c[m].score;
                    break;
                }
            for (int j = k - 1; j >= 0; --j)
                if (c[j].score > b) {
                    if (c[j].score - b < *gap) *gap = c[j].score - b;
                    break;
                }
        }
        int *kept = (int *)malloc(sizeof(int) * (size_t)k);
        for (int j = 0; j < k; ++j) kept[j] = c[j].idx;
        qsort(kept, (size_t)k, sizeof(int), or_int_cmp);
        lvl = (or_state *)malloc(sizeof(or_state) * (size_t)k);
        R = (double *)malloc(sizeof(double) * (size_t)k);
        for (int j = 0; j < k; ++j) {
            lvl[j] = ch[kept[j]];
            R[j] = Rc[kept[j]];
        }
        cnt = k;
        free(kept);
        free(c);
        free(ch);
        free(Rc);
        free(mq);
    }
    /* d == 1: the depth-1 node is the leaf */
    double q[64];
    or_q_of_state(&lvl[0], W, A, q);
    double v = R[0] + gamma * or_maxv(q, A);
    free(lvl);
    free(R);
    return v;
}

int or_search_pruned(const or_state *roots, int n, const float *W, int A, int d, double gamma, double corr,
                     int exact_gev, int keep, int *actions, double *values, double *diag) {
    if (A < 1 || A > 64 || d < 0 || n < 0 || keep < 1) return -1;
    for (int i = 0; i < n; ++i) {
        double q0[64], V[64], delta[64], r0[64];
        double *val = values + (size_t)i * A;
        double *dg = diag ? diag + (size_t)i * (4 * A + 5) : NULL;
        or_q_of_state(&roots[i], W, A, q0);
        int pi_o = or_argmax_lowest(q0, A);
        double gap = INFINITY;
        if (d == 0) {
            for (int a = 0; a < A; ++a) val[a] = q0[a];
            actions[i] = pi_o;
            if (dg) {
                for (int a = 0; a < A; ++a) { dg[a] = q0[a]; dg[A + a] = q0[a]; dg[2 * A + a] = 0; dg[3 * A + a] = 0; }
                dg[4 * A] = pi_o; dg[4 * A + 1] = 0; dg[4 * A + 2] = 0; dg[4 * A + 3] = 0; dg[4 * A + 4] = gap;
            }
            continue;
        }
        for (int a = 0; a < A; ++a) {
            or_state s1;
            int r = or_env_step(&roots[i], a, &s1);
            double q1[64];
            or_q_of_state(&s1, W, A, q1);
            r0[a] = (double)r;
            delta[a] = (double)r + gamma * or_maxv(q1, A) - q0[a];
            V[a] = or_pruned_subtree(&s1, (double)r, W, A, d, gamma, keep, &gap);
        }
        double delta_o = fabs(delta[pi_o]), delta_e = 0.0;
        if (A > 1) {
            for (int a = 0; a < A; ++a)
                if (a != pi_o) delta_e += fabs(delta[a]);
            delta_e /= (double)(A - 1);
        }
        double B = exact_gev ? or_bellman_penalty_exact(delta_e, delta_o, A, d)
                             : or_bellman_penalty(delta_e, delta_o, A, d);
        double gd = pow(gamma, (double)d);
        for (int a = 0; a < A; ++a) val[a] = (a == pi_o) ? V[a] : V[a] - gd * corr * B;
        actions[i] = or_argmax_lowest(val, A);
        if (dg) {
            for (int a = 0; a < A; ++a) { dg[a] = q0[a]; dg[A + a] = V[a]; dg[2 * A + a] = delta[a]; dg[3 * A + a] = r0[a]; }
            dg[4 * A] = pi_o; dg[4 * A + 1] = delta_o; dg[4 * A + 2] = delta_e; dg[4 * A + 3] = B;
            dg[4 * A + 4] = gap;
        }
    }
    return 0;
}
