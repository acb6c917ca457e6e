/*
 * CPU oracle for the MRIP hot path -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
 * (including `bench.py --impl reference`) may load this library.  The CUDA
 * path shares no code, header, table or constant generator with it.
 *
 * Method: Multiple Replications In Parallel (MRIP) -- the same stochastic
 * model run with independent random sources, results averaged and turned
 * into a CLT confidence interval (paper, Section 1 "Introduction").  Every
 * replication here is the plain sequential recurrence, FP64, compiled with
 * -ffp-contract=off, one replication at a time, no blocking or fusion.
 *
 * Random source.  The paper used L'Ecuyer's Tausworthe generator split by
 * random spacing (Section 5).  This engine instead keys a counter-based
 * Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) on (seed, design point, replication,
 * step), so any replication can be recomputed alone.  Counter layout:
 *   c0 = sub-block index inside a step, c1 = step index,
 *   c2 = replication index, c3 = (tag << 24) | design-point index,
 *   key = (seed low 32 bits, seed high 32 bits).
 * Tags: 0 simulation, 1 lattice initial state, 2 control-mean runs,
 *       3 network initialisation, 4 minibatch order, 5 and 6 growth and
 *       lightning gaps of the skip-sampled forest fire.
 *
 * Parity pins live in tests/test_oracle_*.py.  Nothing here is "parity
 * unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the SC'11 definition.                        */
/* One round: the two 32x32->64 products of (M0, c0) and (M1, c2) are formed,
 * their high halves are xored with the other two counter words and the
 * round key, and the low halves move into positions 1 and 3.  Between
 * rounds the key is bumped by the two Weyl constants.                      */
/* ------------------------------------------------------------------------ */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += OR_PHILOX_W0;
            k1 += OR_PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)(prod1 & 0xFFFFFFFFu);
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)(prod0 & 0xFFFFFFFFu);
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Draw the four words of block (c0, c1) of replication `rep` of design point
 * `dp` under `tag`. */
static void or_block(uint64_t seed, uint32_t tag, uint32_t dp, uint32_t rep,
                     uint32_t c1, uint32_t c0, uint32_t out[4])
{
    uint32_t ctr[4];
    uint32_t key[2];
    ctr[0] = c0;
    ctr[1] = c1;
    ctr[2] = rep;
    ctr[3] = (tag << 24) | dp;
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, out);
}

/* 53-bit uniform on [0, 1): the top 53 bits of the 64-bit word hi:lo, scaled
 * by 2^-53.  Exact in double. */
double or_u53(uint32_t lo, uint32_t hi)
{
    uint64_t bits = ((uint64_t)hi << 32) | (uint64_t)lo;
    uint64_t top = bits >> 11;
    return ldexp((double)top, -53);
}

/* Exponential variate by inversion: -log(1 - u) / rate.  1 - u is exact for u
 * on the 2^-53 grid; log is the C library's, the divide is IEEE. */
double or_expo(double u, double rate)
{
    double one_minus_u = 1.0 - u;
    return -log(one_minus_u) / rate;
}

/* Bernoulli threshold: an event of probability p happens iff a uniform
 * 32-bit word w satisfies w < T(p) = floor(p * 2^32).  p in [0, 1). */
uint32_t or_threshold(double p)
{
    double scaled = ldexp(p, 32);
    return (uint32_t)floor(scaled);
}

/* ------------------------------------------------------------------------ */
/* M/M/1 queue (paper, Section 5.1, second model): per client an arrival gap
 * and a service time are drawn; outputs are the average idle time, the
 * average time in queue and the average time in the system.               */
/*                                                                          */
/* Client n (n = 0..N-1) uses block (c0 = 0, c1 = n): words (0,1) give the
 * service time S_n ~ Exp(mu), words (2,3) the gap A_{n+1} ~ Exp(lambda) to
 * the next arrival.  The system starts empty: W_0 = 0.  Lindley:
 *   V_n = W_n + S_n          (time in system of client n)
 *   t_n = V_n - A_{n+1}
 *   W_{n+1} = max(0, t_n),   idle_n = max(0, -t_n)
 * Outputs: mean of W_n, of idle_n and of V_n over n < N.                   */
/* ------------------------------------------------------------------------ */
void or_mm1_rep(double lambda, double mu, int64_t n_clients, uint64_t seed,
                uint32_t dp, uint32_t rep, double out[3])
{
    double w = 0.0;
    double sum_wait = 0.0, sum_idle = 0.0, sum_system = 0.0;
    for (int64_t n = 0; n < n_clients; ++n) {
        uint32_t blk[4];
        or_block(seed, 0u, dp, rep, (uint32_t)n, 0u, blk);
        double s = or_expo(or_u53(blk[0], blk[1]), mu);
        double a = or_expo(or_u53(blk[2], blk[3]), lambda);
        sum_wait += w;
        double v = w + s;
        sum_system += v;
        double t = v - a;
        sum_idle += (t < 0.0) ? -t : 0.0;
        w = (t > 0.0) ? t : 0.0;
    }
    out[0] = sum_wait / (double)n_clients;
    out[1] = sum_idle / (double)n_clients;
    out[2] = sum_system / (double)n_clients;
}

void or_mm1_batch(const double *dps /* n_dp x 2: lambda, mu */, int64_t n_items,
                  const int32_t *dp_idx, const int64_t *rep_idx, int64_t n_clients,
                  uint64_t seed, double *wait, double *idle, double *system)
{
    for (int64_t i = 0; i < n_items; ++i) {
        double o[3];
        int32_t d = dp_idx[i];
        or_mm1_rep(dps[2 * d], dps[2 * d + 1], n_clients, seed, (uint32_t)d,
                   (uint32_t)rep_idx[i], o);
        wait[i] = o[0];
        idle[i] = o[1];
        system[i] = o[2];
    }
}

/* ------------------------------------------------------------------------ */
/* Three-station tandem of M/M/1 queues (FIFO, infinite buffers, all empty at
 * the start) -- the learned-control-variate workload.                      */
/*                                                                          */
/* Client n uses block (c0 = 0, c1 = n): words (0,1) -> gap A_n ~ Exp(lambda)
 * (A_0 is the first arrival time), words (2,3) -> S_{n,1} ~ Exp(mu1); block
 * (c0 = 1, c1 = n): words (0,1) -> S_{n,2}, words (2,3) -> S_{n,3}.
 * With D_{n,j} the departure of client n from station j and a_n its arrival,
 * D_{n,j} = max(D_{n-1,j}, D_{n,j-1}) + S_{n,j}.  Written relative to the
 * arrival, V_{n,j} = D_{n,j} - a_n:
 *   V_{n,0} = 0,  V_{-1,j} = -inf,
 *   V_{n,j} = max(V_{n-1,j} - A_n, V_{n,j-1}) + S_{n,j}
 * (same recurrence, no large absolute clock).  Sojourn_n = V_{n,3};
 * Y = mean over n < N.  Features: lambda, mu1, mu2, mu3 and the means over
 * n < min(N, window) of A_n, S_{n,1}, S_{n,2}, S_{n,3}.                    */
/* ------------------------------------------------------------------------ */
void or_tandem3_rep(const double par[4], int64_t n_clients, int64_t window,
                    uint64_t seed, uint32_t tag, uint32_t dp, uint32_t rep,
                    double *y_out, double feat[8])
{
    double v1 = -INFINITY, v2 = -INFINITY, v3 = -INFINITY;
    double sum_y = 0.0;
    double sum_a = 0.0, sum_s1 = 0.0, sum_s2 = 0.0, sum_s3 = 0.0;
    int64_t w_len = (n_clients < window) ? n_clients : window;
    for (int64_t n = 0; n < n_clients; ++n) {
        uint32_t b0[4], b1[4];
        or_block(seed, tag, dp, rep, (uint32_t)n, 0u, b0);
        or_block(seed, tag, dp, rep, (uint32_t)n, 1u, b1);
        double a = or_expo(or_u53(b0[0], b0[1]), par[0]);
        double s1 = or_expo(or_u53(b0[2], b0[3]), par[1]);
        double s2 = or_expo(or_u53(b1[0], b1[1]), par[2]);
        double s3 = or_expo(or_u53(b1[2], b1[3]), par[3]);
        double q;
        q = v1 - a;
        v1 = ((q > 0.0) ? q : 0.0) + s1;
        q = v2 - a;
        v2 = ((q > v1) ? q : v1) + s2;
        q = v3 - a;
        v3 = ((q > v2) ? q : v2) + s3;
        sum_y += v3;
        if (n < w_len) {
            sum_a += a;
            sum_s1 += s1;
            sum_s2 += s2;
            sum_s3 += s3;
        }
    }
    *y_out = sum_y / (double)n_clients;
    feat[0] = par[0];
    feat[1] = par[1];
    feat[2] = par[2];
    feat[3] = par[3];
    feat[4] = sum_a / (double)w_len;
    feat[5] = sum_s1 / (double)w_len;
    feat[6] = sum_s2 / (double)w_len;
    feat[7] = sum_s3 / (double)w_len;
}

void or_tandem3_batch(const double *dps /* n_dp x 4 */, int64_t n_items,
                      const int32_t *dp_idx, const int64_t *rep_idx,
                      int64_t n_clients, int64_t window, uint64_t seed, uint32_t tag,
                      double *y, double *feat /* n_items x 8 */)
{
    for (int64_t i = 0; i < n_items; ++i) {
        int32_t d = dp_idx[i];
        or_tandem3_rep(dps + 4 * d, n_clients, window, seed, tag, (uint32_t)d,
                       (uint32_t)rep_idx[i], &y[i], feat + 8 * i);
    }
}

/* ------------------------------------------------------------------------ */
/* Stochastic forest-fire cellular automaton (Drossel-Schwabl), L x L
 * periodic lattice, states 0 empty / 1 tree / 2 burning, cell i = y*L + x.
 * Initial state: cell i is a tree iff word (i % 4) of block (c0 = i/4, c1 = 0)
 * under tag 1 is below T(density); otherwise empty; nothing burns.
 * Step t = 1..T, synchronous, from the previous state only, with word
 * w = word (i % 4) of block (c0 = i/4, c1 = t) under tag 0:
 *   burning -> empty;
 *   tree -> burning if any of its 4 von Neumann neighbours burns,
 *           else burning iff w < T(p_lightning), else stays a tree;
 *   empty -> tree iff w < T(p_grow).
 * Output: number of burning cells after each step (T values).             */
/* ------------------------------------------------------------------------ */
int or_forest_fire_rep(int32_t L, int32_t n_steps, double p_grow, double p_light,
                       double density, uint64_t seed, uint32_t dp, uint32_t rep,
                       const uint8_t *init_state /* L*L or NULL */,
                       int32_t *counts /* n_steps */, uint8_t *final_state /* L*L or NULL */)
{
    int64_t n_cells = (int64_t)L * L;
    uint8_t *cur = (uint8_t *)malloc((size_t)n_cells);
    uint8_t *nxt = (uint8_t *)malloc((size_t)n_cells);
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return -1;
    }
    uint32_t t_grow = or_threshold(p_grow);
    uint32_t t_light = or_threshold(p_light);
    uint32_t t_dens = or_threshold(density);
    uint32_t blk[4];

    if (init_state) {
        memcpy(cur, init_state, (size_t)n_cells);
    } else {
        for (int64_t i = 0; i < n_cells; ++i) {
            if (i % 4 == 0)
                or_block(seed, 1u, dp, rep, 0u, (uint32_t)(i / 4), blk);
            cur[i] = (blk[i % 4] < t_dens) ? 1 : 0;
        }
    }

    for (int32_t t = 1; t <= n_steps; ++t) {
        int32_t burning = 0;
        for (int32_t y = 0; y < L; ++y) {
            for (int32_t x = 0; x < L; ++x) {
                int64_t i = (int64_t)y * L + x;
                if (i % 4 == 0)
                    or_block(seed, 0u, dp, rep, (uint32_t)t, (uint32_t)(i / 4), blk);
                uint32_t w = blk[i % 4];
                uint8_t s = cur[i];
                uint8_t ns;
                if (s == 2) {
                    ns = 0;
                } else if (s == 1) {
                    int32_t up = (y + L - 1) % L, down = (y + 1) % L;
                    int32_t left = (x + L - 1) % L, right = (x + 1) % L;
                    int fire_near = cur[(int64_t)up * L + x] == 2 ||
                                    cur[(int64_t)down * L + x] == 2 ||
                                    cur[(int64_t)y * L + left] == 2 ||
                                    cur[(int64_t)y * L + right] == 2;
                    if (fire_near)
                        ns = 2;
                    else if (w < t_light)
                        ns = 2;
                    else
                        ns = 1;
                } else {
                    ns = (w < t_grow) ? 1 : 0;
                }
                nxt[i] = ns;
                if (ns == 2)
                    ++burning;
            }
        }
        counts[t - 1] = burning;
        uint8_t *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (final_state)
        memcpy(final_state, cur, (size_t)n_cells);
    free(cur);
    free(nxt);
    return 0;
}

int or_forest_fire_batch(int32_t L, int32_t n_steps, const double *dps /* n_dp x 2 */,
                         double density, int64_t n_items, const int32_t *dp_idx,
                         const int64_t *rep_idx, uint64_t seed,
                         int32_t *counts /* n_items x n_steps */)
{
    for (int64_t i = 0; i < n_items; ++i) {
        int32_t d = dp_idx[i];
        int rc = or_forest_fire_rep(L, n_steps, dps[2 * d], dps[2 * d + 1], density, seed,
                                    (uint32_t)d, (uint32_t)rep_idx[i], NULL,
                                    counts + (int64_t)n_steps * i, NULL);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Forest fire with skip-sampled events (an engine variant of the automaton
 * above; same rules, same initial state from tag 1).  Instead of one word
 * per cell, each step draws two event sets over the cells i = 0 .. L^2 - 1:
 * growth events (each cell independently with probability p_grow) and
 * lightning events (probability p_light).  An empty cell in the growth set
 * becomes a tree; a tree with no burning neighbour in the lightning set
 * ignites.  Per cell and step this is the same law as the per-cell model.
 *
 * Event set of probability p (Bernoulli trials over the cells in index
 * order, sampled by the gaps between successes): with mu = -log1p(-p), gap
 * j (j = 0, 1, ...) is K_j = floor(E_j / mu), E_j = -log(1 - u) the
 * exponential variate of or_expo, u from words 2(j mod 2), 2(j mod 2) + 1
 * of block (c0 = j div 2, c1 = t) under tag 5 (growth) or 6 (lightning);
 * P(K_j >= k) = (1 - p)^k.  Events sit at pos_0 = K_0 and
 * pos_j = pos_{j-1} + 1 + K_j while below L^2.  p = 0: no events.
 *
 * Where floating point decides the integer K_j, a result within a few ulps
 * of an integer could round either way on another machine; such draws are
 * counted in *near_ties (the tests compare only replications with none). */
/* ------------------------------------------------------------------------ */
static void or_skip_events(uint8_t *ev, int64_t n_cells, double p, uint32_t tag, uint64_t seed,
                           uint32_t dp, uint32_t rep, uint32_t t, int64_t *near_ties)
{
    memset(ev, 0, (size_t)n_cells);
    if (!(p > 0.0))
        return;
    double mu = -log1p(-p);
    int64_t pos = -1;
    uint32_t blk[4];
    for (uint32_t j = 0;; ++j) {
        if ((j & 1u) == 0)
            or_block(seed, tag, dp, rep, t, j >> 1, blk);
        double x = or_expo(or_u53(blk[2 * (j & 1u)], blk[2 * (j & 1u) + 1]), mu);
        double nearest = floor(x + 0.5);  /* floor(x) is ambiguous only near 1, 2, ... */
        if (nearest >= 1.0 && fabs(x - nearest) <= ldexp(x, -48) + ldexp(1.0 / mu, -50))
            ++*near_ties;
        /* the next event is pos + 1 + floor(x); stop once it is off the lattice */
        if (x >= (double)(n_cells - pos - 1))
            break;
        pos += 1 + (int64_t)x;
        ev[pos] = 1;
    }
}

int or_forest_fire_skip_rep(int32_t L, int32_t n_steps, double p_grow, double p_light,
                            double density, uint64_t seed, uint32_t dp, uint32_t rep,
                            const uint8_t *init_state /* L*L or NULL */,
                            int32_t *counts /* n_steps */, uint8_t *final_state /* L*L or NULL */,
                            int64_t *near_ties)
{
    int64_t n_cells = (int64_t)L * L;
    uint8_t *cur = (uint8_t *)malloc((size_t)n_cells);
    uint8_t *nxt = (uint8_t *)malloc((size_t)n_cells);
    uint8_t *grow = (uint8_t *)malloc((size_t)n_cells);
    uint8_t *light = (uint8_t *)malloc((size_t)n_cells);
    if (!cur || !nxt || !grow || !light) {
        free(cur);
        free(nxt);
        free(grow);
        free(light);
        return -1;
    }
    *near_ties = 0;
    uint32_t t_dens = or_threshold(density);
    uint32_t blk[4];
    if (init_state) {
        memcpy(cur, init_state, (size_t)n_cells);
    } else {
        for (int64_t i = 0; i < n_cells; ++i) {
            if (i % 4 == 0)
                or_block(seed, 1u, dp, rep, 0u, (uint32_t)(i / 4), blk);
            cur[i] = (blk[i % 4] < t_dens) ? 1 : 0;
        }
    }
    for (int32_t t = 1; t <= n_steps; ++t) {
        or_skip_events(grow, n_cells, p_grow, 5u, seed, dp, rep, (uint32_t)t, near_ties);
        or_skip_events(light, n_cells, p_light, 6u, seed, dp, rep, (uint32_t)t, near_ties);
        int32_t burning = 0;
        for (int32_t y = 0; y < L; ++y) {
            for (int32_t x = 0; x < L; ++x) {
                int64_t i = (int64_t)y * L + x;
                uint8_t s = cur[i];
                uint8_t ns;
                if (s == 2) {
                    ns = 0;
                } else if (s == 1) {
                    int32_t up = (y + L - 1) % L, down = (y + 1) % L;
                    int32_t left = (x + L - 1) % L, right = (x + 1) % L;
                    int fire_near = cur[(int64_t)up * L + x] == 2 ||
                                    cur[(int64_t)down * L + x] == 2 ||
                                    cur[(int64_t)y * L + left] == 2 ||
                                    cur[(int64_t)y * L + right] == 2;
                    ns = (fire_near || light[i]) ? 2 : 1;
                } else {
                    ns = grow[i] ? 1 : 0;
                }
                nxt[i] = ns;
                if (ns == 2)
                    ++burning;
            }
        }
        counts[t - 1] = burning;
        uint8_t *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (final_state)
        memcpy(final_state, cur, (size_t)n_cells);
    free(cur);
    free(nxt);
    free(grow);
    free(light);
    return 0;
}

int or_forest_fire_skip_batch(int32_t L, int32_t n_steps, const double *dps /* n_dp x 2 */,
                              double density, int64_t n_items, const int32_t *dp_idx,
                              const int64_t *rep_idx, uint64_t seed,
                              int32_t *counts /* n_items x n_steps */, int64_t *near_ties)
{
    for (int64_t i = 0; i < n_items; ++i) {
        int32_t d = dp_idx[i];
        int rc = or_forest_fire_skip_rep(L, n_steps, dps[2 * d], dps[2 * d + 1], density, seed,
                                         (uint32_t)d, (uint32_t)rep_idx[i], NULL,
                                         counts + (int64_t)n_steps * i, NULL, near_ties + i);
        if (rc != 0)
            return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exit time of a simple random walk on Z^2 from the origin out of the L1
 * ball |x| + |y| < R (the uneven-length workload; it adapts the paper's
 * random-walk model of Section 5.1 to a stopping time).  Move m (m = 0, 1,
 * ...) reads the 2-bit field k = m & 63 of block (c0 = 0, c1 = m >> 6):
 * word k >> 4, bits 2(k & 15) and 2(k & 15) + 1.  Field 0: +x, 1: -x,
 * 2: +y, 3: -y.  Output: tau = number of moves made when |x| + |y| first
 * reaches R; -1 if max_steps moves did not reach it.                       */
/* ------------------------------------------------------------------------ */
int64_t or_walk_rep(int64_t radius, uint64_t seed, uint32_t dp, uint32_t rep, int64_t max_steps)
{
    int64_t x = 0, y = 0;
    uint32_t blk[4];
    for (int64_t m = 0; m < max_steps; ++m) {
        if ((m & 63) == 0)
            or_block(seed, 0u, dp, rep, (uint32_t)(m >> 6), 0u, blk);
        int k = (int)(m & 63);
        uint32_t field = (blk[k >> 4] >> (2 * (k & 15))) & 3u;
        if (field == 0)
            x += 1;
        else if (field == 1)
            x -= 1;
        else if (field == 2)
            y += 1;
        else
            y -= 1;
        int64_t norm = (x < 0 ? -x : x) + (y < 0 ? -y : y);
        if (norm >= radius)
            return m + 1;
    }
    return -1;
}

void or_walk_batch(const double *radii /* n_dp */, int64_t n_items, const int32_t *dp_idx,
                   const int64_t *rep_idx, uint64_t seed, int64_t max_steps, int64_t *tau)
{
    for (int64_t i = 0; i < n_items; ++i) {
        int32_t d = dp_idx[i];
        tau[i] = or_walk_rep((int64_t)radii[d], seed, (uint32_t)d, (uint32_t)rep_idx[i],
                             max_steps);
    }
}

/* ------------------------------------------------------------------------ */
/* Student-t quantile for the confidence interval (paper, Section 1: the
 * replication mean is approximately Gaussian by the CLT, which is what the
 * interval rests on; with an estimated variance the interval uses Student's
 * t with n - 1 degrees of freedom).
 *
 * For integer nu the two-sided probability A(t|nu) = P(|T| <= t) has a
 * finite series in theta = atan(t / sqrt(nu)) (Abramowitz & Stegun 26.7.3
 * and 26.7.4):
 *   nu odd:  A = (2/pi) (theta + sin(theta) sum_{k=0}^{(nu-3)/2} a_k cos^{2k+1}(theta)),
 *            a_0 = 1, a_k = a_{k-1} * 2k / (2k + 1)           (nu = 1: A = 2 theta / pi)
 *   nu even: A = sin(theta) sum_{k=0}^{(nu-2)/2} b_k cos^{2k}(theta),
 *            b_0 = 1, b_k = b_{k-1} * (2k - 1) / (2k)
 * The terms are accumulated in double-double (error-free sum and product)
 * because nu reaches 2^17.  The quantile solves (1 + A(t)) / 2 = p by
 * bracketing bisection on t in double, which needs no density.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double hi, lo;
} or_dd;

static or_dd or_dd_add(or_dd a, or_dd b)
{
    double s = a.hi + b.hi;
    double bb = s - a.hi;
    double err = (a.hi - (s - bb)) + (b.hi - bb);
    err += a.lo + b.lo;
    or_dd r;
    r.hi = s + err;
    r.lo = err - (r.hi - s);
    return r;
}

static or_dd or_dd_mul(or_dd a, or_dd b)
{
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e += a.hi * b.lo + a.lo * b.hi;
    or_dd r;
    r.hi = p + e;
    r.lo = e - (r.hi - p);
    return r;
}

static or_dd or_dd_from(double x)
{
    or_dd r;
    r.hi = x;
    r.lo = 0.0;
    return r;
}

/* num / den for small integers, as a double-double */
static or_dd or_dd_ratio(double num, double den)
{
    double q = num / den;
    double rem = fma(-q, den, num); /* exact remainder */
    or_dd r;
    r.hi = q;
    r.lo = rem / den;
    return or_dd_add(or_dd_from(0.0), r);
}

/* a / b for double-doubles: one correction step after the double quotient */
static or_dd or_dd_div(or_dd a, or_dd b)
{
    double q1 = a.hi / b.hi;
    or_dd prod = or_dd_mul(b, or_dd_from(q1));
    or_dd rem = or_dd_add(a, or_dd_from(-prod.hi));
    rem = or_dd_add(rem, or_dd_from(-prod.lo));
    double q2 = rem.hi / b.hi;
    return or_dd_add(or_dd_from(q1), or_dd_from(q2));
}

/* P(|T| <= t) for t >= 0 as a double-double.  cos^2(theta) = nu / (nu + t^2)
 * is formed in double-double because the series raises it to powers up to
 * nu / 2; sin(theta) and theta enter once and are taken in double. */
static or_dd or_t_two_sided(double t, int64_t nu)
{
    double r = sqrt((double)nu + t * t);
    double s = t / r;                    /* sin(theta) */
    double theta = atan2(t, sqrt((double)nu));
    or_dd t2 = or_dd_mul(or_dd_from(t), or_dd_from(t));
    or_dd den = or_dd_add(or_dd_from((double)nu), t2);
    or_dd c2 = or_dd_div(or_dd_from((double)nu), den);
    double c = sqrt(c2.hi + c2.lo);      /* cos(theta), enters once */
    if (nu % 2 == 1) {
        or_dd sum = or_dd_from(0.0);
        if (nu >= 3) {
            or_dd term = or_dd_from(c);
            sum = term;
            for (int64_t k = 1; k <= (nu - 3) / 2; ++k) {
                term = or_dd_mul(term, or_dd_ratio(2.0 * (double)k, 2.0 * (double)k + 1.0));
                term = or_dd_mul(term, c2);
                sum = or_dd_add(sum, term);
            }
        }
        or_dd inner = or_dd_add(or_dd_from(theta), or_dd_mul(or_dd_from(s), sum));
        return or_dd_mul(inner, or_dd_ratio(2.0, M_PI));
    } else {
        or_dd term = or_dd_from(1.0);
        or_dd sum = term;
        for (int64_t k = 1; k <= (nu - 2) / 2; ++k) {
            term = or_dd_mul(term, or_dd_ratio(2.0 * (double)k - 1.0, 2.0 * (double)k));
            term = or_dd_mul(term, c2);
            sum = or_dd_add(sum, term);
        }
        return or_dd_mul(or_dd_from(s), sum);
    }
}

/* CDF of Student's t with nu degrees of freedom, as a double. */
double or_t_cdf(double t, int64_t nu)
{
    if (nu < 1)
        return NAN;
    double at = fabs(t);
    or_dd a = or_t_two_sided(at, nu);
    or_dd half = or_dd_from(0.5);
    or_dd upper_tail = or_dd_mul(half, or_dd_add(or_dd_from(1.0), or_dd_from(-a.hi)));
    upper_tail = or_dd_add(upper_tail, or_dd_mul(half, or_dd_from(-a.lo)));
    if (t >= 0)
        return 1.0 - (upper_tail.hi + upper_tail.lo);
    return upper_tail.hi + upper_tail.lo;
}

/* Upper-tail probability 1 - F(t) for t >= 0, computed without the
 * cancellation of 1 - F. */
static double or_t_upper(double t, int64_t nu)
{
    or_dd a = or_t_two_sided(t, nu);
    or_dd one_minus = or_dd_add(or_dd_from(1.0), or_dd_from(-a.hi));
    one_minus = or_dd_add(one_minus, or_dd_from(-a.lo));
    return 0.5 * (one_minus.hi + one_minus.lo);
}

/* Critical value of the two-sided interval at confidence `conf`: the t > 0
 * with P(T > t) = (1 - conf) / 2, for conf in (0, 1). */
double or_t_crit(double conf, int64_t nu)
{
    if (nu < 1 || !(conf > 0.0) || !(conf < 1.0))
        return NAN;
    double target = (1.0 - conf) / 2.0;
    double lo = 0.0, hi = 1.0;
    while (or_t_upper(hi, nu) > target)
        hi *= 2.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi)
            break;
        if (or_t_upper(mid, nu) > target)
            lo = mid;
        else
            hi = mid;
    }
    /* the end of the final bracket whose tail is closer to the target */
    double elo = fabs(or_t_upper(lo, nu) - target);
    double ehi = fabs(or_t_upper(hi, nu) - target);
    return (elo < ehi) ? lo : hi;
}

/* p-quantile for p in (0.5, 1): the critical value with conf = 2p - 1. */
double or_t_quantile(double p, int64_t nu)
{
    if (!(p > 0.5) || !(p < 1.0))
        return NAN;
    return or_t_crit(2.0 * p - 1.0, nu);
}

/* ------------------------------------------------------------------------ */
/* Array helpers for the Python side (no arithmetic beyond the above).      */
/* ------------------------------------------------------------------------ */
void or_philox_batch(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i)
        or_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

void or_expo_batch(int64_t n, const uint32_t *lo, const uint32_t *hi, const double *rate,
                   double *u_out, double *e_out)
{
    for (int64_t i = 0; i < n; ++i) {
        double u = or_u53(lo[i], hi[i]);
        u_out[i] = u;
        e_out[i] = or_expo(u, rate[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Area walk: the paper's random-walk model (Section 5.1, third model, after
 * Vattulainen & Ala-Nissila): a walker on a map split into 30 areas; at the
 * end the walkers are counted per area.  Reading (the paper gives no sizes):
 * a 60 x 50 periodic map, areas of 10 x 10 cells numbered a = x/10 + 6 (y/10),
 * start at (30, 25).  Move m reads the same 2-bit field as the L1 walk:
 * field m mod 64 of block (c0 = 0, c1 = m div 64); 0:+x 1:-x 2:+y 3:-y.
 * After every move the visit count of the walker's area is incremented.
 * Outputs: the final area and the 30 visit counts.                        */
/* ------------------------------------------------------------------------ */
#define OR_AW_W 60
#define OR_AW_H 50
#define OR_AW_CELL 10
#define OR_AW_AREAS 30

void or_area_walk_rep(int32_t n_steps, uint64_t seed, uint32_t rep, int32_t *final_area,
                      int32_t visits[30])
{
    int32_t x = OR_AW_W / 2, y = OR_AW_H / 2;
    uint32_t blk[4];
    for (int a = 0; a < OR_AW_AREAS; ++a)
        visits[a] = 0;
    for (int32_t m = 0; m < n_steps; ++m) {
        if ((m & 63) == 0)
            or_block(seed, 0u, 0u, rep, (uint32_t)(m >> 6), 0u, blk);
        int k = m & 63;
        uint32_t field = (blk[k >> 4] >> (2 * (k & 15))) & 3u;
        if (field == 0)
            x = (x + 1) % OR_AW_W;
        else if (field == 1)
            x = (x + OR_AW_W - 1) % OR_AW_W;
        else if (field == 2)
            y = (y + 1) % OR_AW_H;
        else
            y = (y + OR_AW_H - 1) % OR_AW_H;
        visits[x / OR_AW_CELL + (OR_AW_W / OR_AW_CELL) * (y / OR_AW_CELL)] += 1;
    }
    *final_area = x / OR_AW_CELL + (OR_AW_W / OR_AW_CELL) * (y / OR_AW_CELL);
}

void or_area_walk_batch(int64_t n_items, const int64_t *rep_idx, int32_t n_steps, uint64_t seed,
                        int32_t *final_area, int32_t *visits /* n_items x 30 */)
{
    for (int64_t i = 0; i < n_items; ++i)
        or_area_walk_rep(n_steps, seed, (uint32_t)rep_idx[i], &final_area[i], visits + 30 * i);
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo pi (paper, Section 5.1, first model): random points in the
 * unit square, counted when they fall in the quarter disc; pi is estimated
 * by 4 hits / draws.  Draw k uses words 2(k mod 2) and 2(k mod 2)+1 of block
 * (c0 = 0, c1 = k div 2) as integer coordinates x, y in [0, 2^32); the
 * point is inside iff x^2 + y^2 < 2^64 (exact in integers).  Output: hits. */
/* ------------------------------------------------------------------------ */
int64_t or_pi_rep(int64_t n_draws, uint64_t seed, uint32_t rep)
{
    int64_t hits = 0;
    uint32_t blk[4];
    for (int64_t k = 0; k < n_draws; ++k) {
        if ((k & 1) == 0)
            or_block(seed, 0u, 0u, rep, (uint32_t)(k >> 1), 0u, blk);
        uint64_t x = blk[2 * (k & 1)], y = blk[2 * (k & 1) + 1];
        uint64_t x2 = x * x, y2 = y * y;
        /* x^2 + y^2 < 2^64  <=>  x^2 <= 2^64 - 1 - y^2 */
        if (x2 <= UINT64_MAX - y2)
            ++hits;
    }
    return hits;
}

void or_pi_batch(int64_t n_items, const int64_t *rep_idx, int64_t n_draws, uint64_t seed,
                 int64_t *hits)
{
    for (int64_t i = 0; i < n_items; ++i)
        hits[i] = or_pi_rep(n_draws, seed, (uint32_t)rep_idx[i]);
}
