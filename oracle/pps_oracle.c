/*
 * pps_oracle.c -- plain FP64 CPU oracle for the passing-point search of the
 * ZJUNlict 2019 team description paper.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are its only callers.  It shares nothing with the CUDA
 * path.  It is written to be read against the paper, not to be fast: every
 * candidate pass recomputes every intercept time, loops run in the order of
 * the definitions, and nothing is blocked, fused or reordered.
 *
 * What the paper fixes and what this file reads into it:
 *
 *  Sec. 4.1  The ball is kicked, slides briefly, then rolls with a small
 *            constant deceleration; the sliding phase is neglected, and
 *            Eq. 1 relates distance d, time t, speed and the rolling
 *            deceleration a.  Eq. 1 is garbled in print; read as
 *            d = v t - a t^2 / 2.  READING: the kick speed is the speed at
 *            which rolling starts (no 5/7 slide factor on this path).
 *  Sec. 4.2  A pass is feasible when no opponent can intercept the ball
 *            (SBIP, cited but not defined).  READING: the ball is sampled
 *            at K points spaced uniformly in distance along the pass line,
 *            k = 1..K (the kick point excluded, the receiver included); an
 *            opponent intercepts at sample k when it can be there no later
 *            than the ball.  The opponent's minimum time is that of a 1-D
 *            bang-bang motion along the line to the sample: full
 *            acceleration amax toward it, speed capped at vmax, starting
 *            from the component of its velocity toward the sample (the
 *            perpendicular component dropped), arriving at any speed.
 *  Sec. 4.3  Score = sum_i w_i x_i (Eq. 3); lengths and angles divided by
 *            their upper bound, times unchanged.  Features used here: shot
 *            angle at the receiver (angle / pi), distance from the receiver
 *            to the opponent goal (/ field diagonal, counted negatively:
 *            shorter is better) and the intercept-time margin (capped).
 *  Sec. 4.4  Shot angle: the valid angle to the goal given the opponents'
 *            positions.  READING: the largest contiguous part of the goal
 *            mouth's angular interval not covered by any opponent disc.
 *  Sec. 1 / Sec. 4.3  The best pass is the highest score; READING: ties go
 *            to the smallest candidate index.
 *
 * Further sections, each with its readings beside the code:
 *  D   Sec. 4.2 as the paper parameterises it: directions x kick powers
 *      from the ball holder, teammates and opponents searched along every
 *      ball path (the 5/7 slide of Sec. 4.1 applied), Sec. 4.3's features.
 *  D2  Sec. 4.1, Eq. 1-2: the kick power for a receiver and a target.
 *  D3  Sec. 4.4: the shooting decision.
 *  R   Sec. 5.1-5.2: running points -- four ball-dependent zones over the
 *      attacking half, the five criteria of Eq. 4, the supporters' zones.
 */
#include "pps_oracle.h"

#include <math.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- C1: the candidate grid (Sec. 5.1 rasterises at a fixed spacing) ---- */
void pps_oracle_grid(double L, double W, double g, int* nx, int* ny,
                     double* x0, double* y0)
{
    /* Field corners are included: 12 m at 0.1 m gives 121 columns. */
    *nx = (int)lround(L / g) + 1;
    *ny = (int)lround(W / g) + 1;
    *x0 = -0.5 * L;
    *y0 = -0.5 * W;
}

/* ---- C2: ball arrival time (Sec. 4.1, Eq. 1) ---- */
double pps_oracle_ball_time(double s, double v, double a)
{
    /* Rolling from speed v with deceleration a: s(t) = v t - a t^2 / 2.
     * The first time s is reached is the smaller root of a t^2/2 - v t + s,
     * t = (v - sqrt(v^2 - 2 a s)) / a, written here in the algebraically
     * equal form 2 s / (v + sqrt(v^2 - 2 a s)), which also covers a = 0.
     * Past the stopping distance v^2 / (2a) the ball never arrives. */
    double disc = v * v - 2.0 * a * s;
    if (disc < 0.0) return INFINITY;
    return 2.0 * s / (v + sqrt(disc));
}

/* ---- C3: opponent minimum intercept time (Sec. 4.2, SBIP) ---- */
double pps_oracle_intercept_time(double ox, double oy, double ux, double uy,
                                 double px, double py, double vmax,
                                 double amax, double reach)
{
    double dx = px - ox, dy = py - oy;
    double d = sqrt(dx * dx + dy * dy);
    if (d <= reach) return 0.0; /* already within reach */

    /* Velocity component along the line toward the sample point. */
    double w = (ux * dx + uy * dy) / d;
    if (w > vmax) w = vmax;
    if (w < -vmax) w = -vmax;

    /* Distance the centre must cover to come within reach. */
    double dist = d - reach;

    /* Accelerate at amax toward the point until the speed reaches vmax:
     * that takes (vmax - w)/amax and covers (vmax^2 - w^2)/(2 amax). */
    double t_top = (vmax - w) / amax;
    double d_top = (vmax * vmax - w * w) / (2.0 * amax);
    if (dist <= d_top) {
        /* Arrives while still accelerating: w t + amax t^2 / 2 = dist. */
        return (-w + sqrt(w * w + 2.0 * amax * dist)) / amax;
    }
    /* Otherwise cruise the rest at vmax. */
    return t_top + (dist - d_top) / vmax;
}

double pps_oracle_min_intercept(const pps_oracle_state* st, double px,
                                double py, double reach)
{
    double vmax = st->sc[PPS_ORACLE_VMAX], amax = st->sc[PPS_ORACLE_AMAX];
    double T = INFINITY;
    for (int j = 0; j < st->n_opp; ++j) {
        const double* o = st->opp + 4 * j;
        double t = pps_oracle_intercept_time(o[0], o[1], o[2], o[3], px, py,
                                             vmax, amax, reach);
        if (t < T) T = t;
    }
    return T;
}

void pps_oracle_min_intercept_many(const pps_oracle_state* st, int n,
                                   const double* pxy, double reach,
                                   double* out)
{
    for (int i = 0; i < n; ++i)
        out[i] = pps_oracle_min_intercept(st, pxy[2 * i], pxy[2 * i + 1],
                                          reach);
}

/* ---- C4: margin and reachability of one candidate pass ---- */
double pps_oracle_margin(const pps_oracle_state* st, double cx, double cy,
                         double v, double reach, double* T_out,
                         int* reachable)
{
    double bx = st->sc[PPS_ORACLE_BALL_X], by = st->sc[PPS_ORACLE_BALL_Y];
    double a = st->sc[PPS_ORACLE_BALL_DECEL];
    double D = sqrt((cx - bx) * (cx - bx) + (cy - by) * (cy - by));
    int reach_ok = (v * v - 2.0 * a * D >= 0.0);
    if (reachable) *reachable = reach_ok;

    double m = INFINITY;
    int K = st->K;
    for (int k = 1; k <= K; ++k) {
        double f = (double)k / (double)K;
        /* Sample k on the pass line and the distance the ball rolls to it. */
        double px = bx + f * (cx - bx);
        double py = by + f * (cy - by);
        double s = f * D;
        double T = pps_oracle_min_intercept(st, px, py, reach);
        if (T_out) T_out[k - 1] = T;
        if (reach_ok) {
            double tb = pps_oracle_ball_time(s, v, a);
            double diff = T - tb;
            if (diff < m) m = diff;
        }
    }
    /* A ball that stops short arrives at time +inf: margin -inf. */
    return reach_ok ? m : -INFINITY;
}

/* ---- C6: shot angle (Sec. 4.3 feature, Sec. 4.4 "valid angle") ---- */
double pps_oracle_shot_angle(const pps_oracle_state* st, double cx,
                             double cy, double r)
{
    double start;
    return pps_oracle_shot_gap(st, cx, cy, r, &start);
}

/* The shot angle and, in *start, the direction where that gap begins. */
double pps_oracle_shot_gap(const pps_oracle_state* st, double cx, double cy,
                           double r, double* start)
{
    *start = 0.0;
    double gx = 0.5 * st->sc[PPS_ORACLE_FIELD_LEN];
    double hw = 0.5 * st->sc[PPS_ORACLE_GOAL_WIDTH];
    /* READING: no shot from on or behind the goal line. */
    if (cx >= gx) return 0.0;

    /* The mouth spans directions lo..hi (both in (-pi/2, pi/2)). */
    double lo = atan2(-hw - cy, gx - cx);
    double hi = atan2(hw - cy, gx - cx);

    /* Each opponent disc blocks the directions within asin(r/d) of the
     * direction to its centre; a disc containing the receiver blocks all. */
    double s[64], e[64];
    int n = 0;
    for (int j = 0; j < st->n_opp && n < 64; ++j) {
        const double* o = st->opp + 4 * j;
        double dx = o[0] - cx, dy = o[1] - cy;
        double d = sqrt(dx * dx + dy * dy);
        if (d <= r) return 0.0;
        double phi = atan2(dy, dx);
        double half = asin(r / d);
        double a0 = phi - half, a1 = phi + half;
        if (a1 <= lo || a0 >= hi) continue; /* misses the mouth */
        s[n] = a0 < lo ? lo : a0;
        e[n] = a1 > hi ? hi : a1;
        ++n;
    }
    /* Sort the blocked intervals by start (insertion sort), then sweep. */
    for (int i = 1; i < n; ++i) {
        double si = s[i], ei = e[i];
        int k = i - 1;
        while (k >= 0 && s[k] > si) {
            s[k + 1] = s[k];
            e[k + 1] = e[k];
            --k;
        }
        s[k + 1] = si;
        e[k + 1] = ei;
    }
    double best = 0.0, cur = lo;
    for (int i = 0; i < n; ++i) {
        if (s[i] > cur && s[i] - cur > best) {
            best = s[i] - cur;
            *start = cur;
        }
        if (e[i] > cur) cur = e[i];
    }
    if (hi - cur > best) {
        best = hi - cur;
        *start = cur;
    }
    return best;
}

/* ---- C5: value function (Sec. 4.3, Eq. 3) ---- */
double pps_oracle_score(const pps_oracle_state* st, const double* prm,
                        double cx, double cy, double margin)
{
    const double pi = 3.14159265358979323846;
    double L = st->sc[PPS_ORACLE_FIELD_LEN], W = st->sc[PPS_ORACLE_FIELD_WID];
    double theta = pps_oracle_shot_angle(st, cx, cy,
                                         prm[PPS_ORACLE_ROBOT_RADIUS]);
    double gdx = 0.5 * L - cx, gdy = 0.0 - cy;
    double dist_goal = sqrt(gdx * gdx + gdy * gdy);
    double diag = sqrt(L * L + W * W);
    double mcap = margin < prm[PPS_ORACLE_MARGIN_CAP]
                      ? margin
                      : prm[PPS_ORACLE_MARGIN_CAP];
    return prm[PPS_ORACLE_W_ANGLE] * theta / pi
         - prm[PPS_ORACLE_W_DIST] * dist_goal / diag
         + prm[PPS_ORACLE_W_MARGIN] * mcap;
}

/* ---- C1..C7 for one state ---- */
static void search_one(const pps_oracle_state* st, double g, int nx, int ny,
                       double x0, double y0, const double* speeds, int V,
                       const double* prm, int64_t* best_idx,
                       double* best_score, double* best_margin,
                       int64_t* n_feasible, uint8_t* feas, double* marg,
                       double* score, double* T, int kstride)
{
    int64_t P = (int64_t)nx * ny;
    double bx = st->sc[PPS_ORACLE_BALL_X], by = st->sc[PPS_ORACLE_BALL_Y];
    double reach = prm[PPS_ORACLE_REACH_RADIUS];
    int64_t bi = -1;
    double bs = -INFINITY, bm = -INFINITY;
    int64_t nf = 0;

    for (int v = 0; v < V; ++v) {
        for (int iy = 0; iy < ny; ++iy) {
            for (int ix = 0; ix < nx; ++ix) {
                int64_t p = (int64_t)iy * nx + ix;
                int64_t idx = (int64_t)v * P + p;
                double cx = x0 + ix * g, cy = y0 + iy * g;
                double D = sqrt((cx - bx) * (cx - bx) + (cy - by) * (cy - by));
                int reachable = 0;
                double* Tk = (T && v == 0) ? T + p * kstride : NULL;
                double m = pps_oracle_margin(st, cx, cy, speeds[v], reach, Tk,
                                             &reachable);
                int ok = reachable && D >= prm[PPS_ORACLE_MIN_PASS_DIST]
                         && m > prm[PPS_ORACLE_TAU_SAFE];
                double sc = ok ? pps_oracle_score(st, prm, cx, cy, m)
                               : -INFINITY;
                if (feas) feas[idx] = (uint8_t)ok;
                if (marg) marg[idx] = m;
                if (score) score[idx] = sc;
                if (ok) {
                    ++nf;
                    /* Highest score; equal scores go to the smaller idx. */
                    if (bi < 0 || sc > bs || (sc == bs && idx < bi)) {
                        bi = idx;
                        bs = sc;
                        bm = m;
                    }
                }
            }
        }
    }
    *best_idx = bi;
    *best_score = bs;
    *best_margin = bm;
    *n_feasible = nf;
}

int pps_oracle_search(int S, const double* sc, const int* n_opp,
                      const int* K, int jstride, const double* opp,
                      double g, int nx, int ny, double x0, double y0,
                      const double* speeds, int V, const double* prm,
                      int64_t* best_idx, double* best_score,
                      double* best_margin, int64_t* n_feasible,
                      uint8_t* feasible, double* margin, double* score,
                      double* T, int kstride, int n_threads)
{
    if (S < 0 || V < 1 || nx < 1 || ny < 1 || !(g > 0.0)) return -1;
    for (int s = 0; s < S; ++s)
        if (n_opp[s] < 0 || n_opp[s] > jstride || K[s] < 1
            || (T && K[s] > kstride))
            return -1;
    int64_t P = (int64_t)nx * ny;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int s = 0; s < S; ++s) {
        pps_oracle_state st;
        st.sc = sc + (int64_t)s * PPS_ORACLE_NSCALAR;
        st.n_opp = n_opp[s];
        st.opp = opp + (int64_t)s * jstride * 4;
        st.K = K[s];
        search_one(&st, g, nx, ny, x0, y0, speeds, V, prm, best_idx + s,
                   best_score + s, best_margin + s, n_feasible + s,
                   feasible ? feasible + (int64_t)s * V * P : NULL,
                   margin ? margin + (int64_t)s * V * P : NULL,
                   score ? score + (int64_t)s * V * P : NULL,
                   T ? T + (int64_t)s * P * kstride : NULL, kstride);
    }
    (void)n_threads;
    return 0;
}

/* ---- D: the paper's own search, directions x kick powers (Sec. 4.2) ---- */

/* READING: the ball rolls from the holder's position b; the path ends where
 * the ball stops or first reaches the field edge, whichever comes first. */
double pps_oracle_dpps_path(const pps_oracle_dpps_state* st, double ux,
                            double uy, double v, int* stopped)
{
    double bx = st->sc[PPS_ORACLE_BALL_X], by = st->sc[PPS_ORACLE_BALL_Y];
    double a = st->sc[PPS_ORACLE_BALL_DECEL];
    double hl = 0.5 * st->sc[PPS_ORACLE_FIELD_LEN];
    double hw = 0.5 * st->sc[PPS_ORACLE_FIELD_WID];
    double s_stop = v * v / (2.0 * a);
    double s_out = INFINITY;
    if (ux > 0.0) s_out = fmin(s_out, (hl - bx) / ux);
    if (ux < 0.0) s_out = fmin(s_out, (-hl - bx) / ux);
    if (uy > 0.0) s_out = fmin(s_out, (hw - by) / uy);
    if (uy < 0.0) s_out = fmin(s_out, (-hw - by) / uy);
    if (s_out < 0.0) s_out = 0.0;
    *stopped = s_stop <= s_out;
    return *stopped ? s_stop : s_out;
}

/* SBIP of a group (Sec. 4.2): the ball's path is searched sample by sample
 * (READING: K samples uniform in distance, the start excluded, as in C4)
 * for the first one a robot of the group can reach no later than the
 * ball; C3 gives each robot's minimum arrival time. */
double pps_oracle_dpps_group(const pps_oracle_dpps_state* st, int n,
                             const double* robots, double ux, double uy,
                             double v, double reach, int* k_out, int* who)
{
    return pps_oracle_dpps_group_margin(st, n, robots, ux, uy, v, reach,
                                        k_out, who, NULL);
}

double pps_oracle_dpps_group_margin(const pps_oracle_dpps_state* st, int n,
                                    const double* robots, double ux,
                                    double uy, double v, double reach,
                                    int* k_out, int* who, double* margin)
{
    if (margin) *margin = INFINITY;
    double bx = st->sc[PPS_ORACLE_BALL_X], by = st->sc[PPS_ORACLE_BALL_Y];
    double a = st->sc[PPS_ORACLE_BALL_DECEL];
    double vmax = st->sc[PPS_ORACLE_VMAX], amax = st->sc[PPS_ORACLE_AMAX];
    int stopped = 0;
    double S = pps_oracle_dpps_path(st, ux, uy, v, &stopped);
    int K = st->K;
    *k_out = 0;
    *who = -1;
    if (n <= 0) return INFINITY;
    for (int k = 1; k <= K; ++k) {
        double s = (double)k / (double)K * S;
        double px = bx + s * ux, py = by + s * uy;
        /* READING: a path that ends by stopping leaves the ball at rest at
         * its last sample, time v / a; any robot gets it there. */
        int last_stop = stopped && k == K;
        double tk = last_stop ? v / a : pps_oracle_ball_time(s, v, a);
        double T = INFINITY;
        int w = -1;
        for (int r = 0; r < n; ++r) {
            const double* o = robots + 4 * r;
            double t = pps_oracle_intercept_time(o[0], o[1], o[2], o[3], px,
                                                 py, vmax, amax, reach);
            if (t < T) {
                T = t;
                w = r;
            }
        }
        /* how far from flipping each searched sample's decision was */
        if (margin && !last_stop && fabs(T - tk) < *margin)
            *margin = fabs(T - tk);
        if (T <= tk || last_stop) {
            *k_out = k;
            *who = w;
            return T <= tk ? tk : T;
        }
    }
    return INFINITY;
}

void pps_oracle_dpps_candidate(const pps_oracle_dpps_state* st,
                               const double* prm, int ndir, int npow, int i,
                               int j, double* out)
{
    const double pi = 3.14159265358979323846;
    double phi = 2.0 * pi * (double)i / (double)ndir;
    double ux = cos(phi), uy = sin(phi);
    double vlo = prm[PPS_ORACLE_D_VLO], vhi = prm[PPS_ORACLE_D_VHI];
    double v0 = npow > 1 ? vlo + (double)j * (vhi - vlo) / (double)(npow - 1)
                         : vlo;
    /* Sec. 4.1: the kick speed drops to 5/7 in a short slide whose distance
     * the paper neglects; the ball then rolls from v = slide * v0. */
    double v = prm[PPS_ORACLE_D_SLIDE] * v0;
    double reach = prm[PPS_ORACLE_D_REACH_RADIUS];
    int k_team, who, k_opp, who_opp;
    double m_team, m_opp;
    double t_team = pps_oracle_dpps_group_margin(st, st->n_team, st->team, ux,
                                                 uy, v, reach, &k_team, &who,
                                                 &m_team);
    double t_opp = pps_oracle_dpps_group_margin(st, st->n_opp, st->opp, ux, uy,
                                                v, reach, &k_opp, &who_opp,
                                                &m_opp);
    /* Sec. 4.3: safe only when the first opponent comes later than the
     * first teammate by more than a threshold. */
    int ok = isfinite(t_team) && (t_opp - t_team > prm[PPS_ORACLE_D_TAU_DELTA]);
    double px = NAN, py = NAN, score = -INFINITY;
    if (k_team > 0) {
        int stopped;
        double S = pps_oracle_dpps_path(st, ux, uy, v, &stopped);
        double s = (double)k_team / (double)st->K * S;
        px = st->sc[PPS_ORACLE_BALL_X] + s * ux;
        py = st->sc[PPS_ORACLE_BALL_Y] + s * uy;
    }
    if (ok) {
        double L = st->sc[PPS_ORACLE_FIELD_LEN], W = st->sc[PPS_ORACLE_FIELD_WID];
        pps_oracle_state os;
        os.sc = st->sc;
        os.n_opp = st->n_opp;
        os.opp = st->opp;
        os.K = st->K;
        double theta = pps_oracle_shot_angle(&os, px, py,
                                             prm[PPS_ORACLE_D_ROBOT_RADIUS]);
        double gx = 0.5 * L - px, gy = -py;
        double dg = sqrt(gx * gx + gy * gy);
        /* READING: the refraction angle of Sec. 4.3 is the turn between the
         * pass direction and the shot direction from the receive point. */
        double refr = 0.0;
        if (dg > 0.0) {
            double c = (ux * gx + uy * gy) / dg;
            refr = acos(c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c));
        }
        double delta = t_opp - t_team;
        double cap = prm[PPS_ORACLE_D_DELTA_CAP];
        score = -prm[PPS_ORACLE_D_W_TIME] * t_team
              + prm[PPS_ORACLE_D_W_ANGLE] * theta / pi
              - prm[PPS_ORACLE_D_W_DIST] * dg / sqrt(L * L + W * W)
              - prm[PPS_ORACLE_D_W_REFR] * refr / pi
              + prm[PPS_ORACLE_D_W_DELTA] * (delta < cap ? delta : cap);
    }
    out[0] = t_team;
    out[1] = t_opp;
    out[2] = (double)k_team;
    out[3] = (double)who;
    out[4] = px;
    out[5] = py;
    out[6] = (double)ok;
    out[7] = score;
    out[8] = m_team;
    out[9] = m_opp;
}

int pps_oracle_dpps_search(int S, const double* sc, const int* n_team,
                           const double* team, const int* n_opp,
                           const double* opp, const int* K, int jstride,
                           int ndir, int npow, const double* prm,
                           int64_t* best_idx, double* best_score,
                           int64_t* n_feasible, uint8_t* feasible,
                           double* score, double* t_team, double* t_opp,
                           int n_threads)
{
    if (S < 0 || ndir < 1 || npow < 1) return -1;
    for (int s = 0; s < S; ++s)
        if (n_team[s] < 0 || n_team[s] > jstride || n_opp[s] < 0
            || n_opp[s] > jstride || K[s] < 1)
            return -1;
    int64_t C = (int64_t)ndir * npow;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int s = 0; s < S; ++s) {
        pps_oracle_dpps_state st;
        st.sc = sc + (int64_t)s * PPS_ORACLE_NSCALAR;
        st.n_team = n_team[s];
        st.team = team + (int64_t)s * jstride * 4;
        st.n_opp = n_opp[s];
        st.opp = opp + (int64_t)s * jstride * 4;
        st.K = K[s];
        int64_t bi = -1, nf = 0;
        double bs = -INFINITY;
        for (int i = 0; i < ndir; ++i)
            for (int j = 0; j < npow; ++j) {
                double out[10];
                pps_oracle_dpps_candidate(&st, prm, ndir, npow, i, j, out);
                int64_t idx = (int64_t)i * npow + j;
                int64_t o = (int64_t)s * C + idx;
                if (feasible) feasible[o] = (uint8_t)out[6];
                if (score) score[o] = out[7];
                if (t_team) t_team[o] = out[0];
                if (t_opp) t_opp[o] = out[1];
                if (out[6] != 0.0) {
                    ++nf;
                    if (bi < 0 || out[7] > bs) {
                        bi = idx;
                        bs = out[7];
                    }
                }
            }
        best_idx[s] = bi;
        best_score[s] = bs;
        n_feasible[s] = nf;
    }
    (void)n_threads;
    return 0;
}

/* ---- D2: passing power (Sec. 4.1, Eq. 1-2) ---- */
void pps_oracle_pass_power(const pps_oracle_dpps_state* st, int receiver,
                           double tx, double ty, double buffer, double slide,
                           double v_lo, double v_hi, double reach,
                           double* out)
{
    double bx = st->sc[PPS_ORACLE_BALL_X], by = st->sc[PPS_ORACLE_BALL_Y];
    double a = st->sc[PPS_ORACLE_BALL_DECEL];
    const double* r = st->team + 4 * receiver;
    /* the receiver's arrival at the target (C3), plus the buffer time */
    double T = pps_oracle_intercept_time(r[0], r[1], r[2], r[3], tx, ty,
                                         st->sc[PPS_ORACLE_VMAX],
                                         st->sc[PPS_ORACLE_AMAX], reach);
    double t = T + buffer;
    double d = sqrt((tx - bx) * (tx - bx) + (ty - by) * (ty - by));
    /* Eq. 1 (read as d = v1 t - a t^2 / 2): the rolling speed that covers d
     * in t.  READING: if that ball would have stopped before t (d < a t^2
     * / 2), the slowest ball that still reaches the target, sqrt(2 a d). */
    double v1 = t > 0.0 ? (d + 0.5 * a * t * t) / t : INFINITY;
    double vmin = sqrt(2.0 * a * d);
    if (v1 < vmin || d < 0.5 * a * t * t) v1 = vmin;
    /* Eq. 2: the kick power; then the robot's limits */
    double v0 = v1 / slide;
    int clamped = 0;
    if (v0 < v_lo) {
        v0 = v_lo;
        clamped = 1;
    }
    if (v0 > v_hi) {
        v0 = v_hi;
        clamped = 1;
    }
    out[0] = v0;
    out[1] = v1;
    out[2] = t;
    out[3] = T;
    out[4] = clamped;
}

/* ---- D3: shooting decision (Sec. 4.4) ---- */
void pps_oracle_shoot(const pps_oracle_dpps_state* st, double cx, double cy,
                      double v_shot, double slide, double theta_min,
                      double tau, double robot_radius, double reach,
                      double* out)
{
    double a = st->sc[PPS_ORACLE_BALL_DECEL];
    double hl = 0.5 * st->sc[PPS_ORACLE_FIELD_LEN];
    pps_oracle_state os;
    os.sc = st->sc;
    os.n_opp = st->n_opp;
    os.opp = st->opp;
    os.K = st->K;
    /* the largest open gap of the mouth and its middle direction */
    double g0 = 0.0;
    double theta = pps_oracle_shot_gap(&os, cx, cy, robot_radius, &g0);
    double dir = g0 + 0.5 * theta;
    double ux = cos(dir), uy = sin(dir);
    double v = slide * v_shot;
    double t_line = INFINITY, t_opp = INFINITY, margin = INFINITY;
    int shoot = 0;
    if (theta > 0.0 && ux > 0.0) {
        /* the ball rolls from (cx, cy) to the goal line x = L/2 */
        double s_line = (hl - cx) / ux;
        double disc = v * v - 2.0 * a * s_line;
        if (disc >= 0.0) {
            t_line = 2.0 * s_line / (v + sqrt(disc));
            /* opponents searched along the shot as in D (K samples) */
            double vmax = st->sc[PPS_ORACLE_VMAX], amax = st->sc[PPS_ORACLE_AMAX];
            for (int k = 1; k <= st->K; ++k) {
                double s = (double)k / (double)st->K * s_line;
                double px = cx + s * ux, py = cy + s * uy;
                double tk = pps_oracle_ball_time(s, v, a);
                double T = INFINITY;
                for (int j = 0; j < st->n_opp; ++j) {
                    const double* o = st->opp + 4 * j;
                    double tj = pps_oracle_intercept_time(o[0], o[1], o[2], o[3],
                                                          px, py, vmax, amax,
                                                          reach);
                    if (tj < T) T = tj;
                }
                if (fabs(T - tk) < margin) margin = fabs(T - tk);
                if (T <= tk) {
                    t_opp = tk;
                    break;
                }
            }
            /* shoot when the gap is wide enough and no opponent gets the
             * ball before it crosses the line by more than tau */
            shoot = theta >= theta_min && (t_opp - t_line > tau || isinf(t_opp));
        }
    }
    out[0] = theta;
    out[1] = dir;
    out[2] = t_line;
    out[3] = t_opp;
    out[4] = shoot;
    out[5] = margin;
}

/* ---- R: running points (Sec. 5.1-5.2) ---- */

/* The point where the segment from p to q first enters the rectangle
 * [x0, x1] x [y0, y1] (Liang-Barsky); returns 0 if it never does. */
static int segment_entry(double px, double py, double qx, double qy,
                         double x0, double x1, double y0, double y1,
                         double* ex, double* ey)
{
    double t0 = 0.0, t1 = 1.0;
    double dx = qx - px, dy = qy - py;
    double p_[4] = {-dx, dx, -dy, dy};
    double q_[4] = {px - x0, x1 - px, py - y0, y1 - py};
    for (int i = 0; i < 4; ++i) {
        if (p_[i] == 0.0) {
            if (q_[i] < 0.0) return 0;
        } else {
            double r = q_[i] / p_[i];
            if (p_[i] < 0.0) {
                if (r > t1) return 0;
                if (r > t0) t0 = r;
            } else {
                if (r < t0) return 0;
                if (r < t1) t1 = r;
            }
        }
    }
    *ex = px + t0 * dx;
    *ey = py + t0 * dy;
    return 1;
}

/* READING: zones I-IV are the attacking half cut at x = L/4 and at the
 * ball's y, kept within +-W/4 so that no zone closes up.  A point within
 * tol of a cut counts as on it (and so in front of it or above it).  No
 * bounds check: the grid's last column may lie a rounding error beyond
 * L/2. */
static int zone_of(const pps_oracle_dpps_state* st, double px, double py,
                   double tol)
{
    double L = st->sc[PPS_ORACLE_FIELD_LEN], W = st->sc[PPS_ORACLE_FIELD_WID];
    double by = st->sc[PPS_ORACLE_BALL_Y];
    double ys = by < -0.25 * W ? -0.25 * W : (by > 0.25 * W ? 0.25 * W : by);
    return (px >= 0.25 * L - tol ? 2 : 0) + (py >= ys - tol ? 1 : 0);
}

/* READING: the cuts and the defence area's edges fall on grid lines at the
 * decimal spacings the paper rasterises with (0.1 m), where the rounding of
 * i g must not decide; a point within g / 1024 of one counts as on it. */
static double edge_tol(const double* prm)
{
    return prm[PPS_ORACLE_R_SPACING] / 1024.0;
}

int pps_oracle_run_zone(const pps_oracle_dpps_state* st, const double* prm,
                        double px, double py)
{
    double L = st->sc[PPS_ORACLE_FIELD_LEN], W = st->sc[PPS_ORACLE_FIELD_WID];
    if (!(px >= 0.0 && px <= 0.5 * L && fabs(py) <= 0.5 * W)) return -1;
    return zone_of(st, px, py, edge_tol(prm));
}

void pps_oracle_run_point(const pps_oracle_dpps_state* st, const double* prm,
                          double px, double py, double* out)
{
    double L = st->sc[PPS_ORACLE_FIELD_LEN], W = st->sc[PPS_ORACLE_FIELD_WID];
    double bx = st->sc[PPS_ORACLE_BALL_X], by = st->sc[PPS_ORACLE_BALL_Y];
    double hw = 0.5 * st->sc[PPS_ORACLE_GOAL_WIDTH];
    double vmax = st->sc[PPS_ORACLE_VMAX], amax = st->sc[PPS_ORACLE_AMAX];
    /* the opponent's defence area: x in [L/2 - depth, L/2], |y| <= width/2 */
    double x0 = 0.5 * L - prm[PPS_ORACLE_R_DEF_DEPTH], x1 = 0.5 * L;
    double y1 = 0.5 * prm[PPS_ORACLE_R_DEF_WIDTH], y0 = -y1;
    /* 1. distance to the opponent's goal, a cost */
    double gx = x1 - px, gy = -py;
    double x_goal = sqrt(gx * gx + gy * gy) / sqrt(L * L + W * W);
    /* 2. distance to the ball: being too close is bad (READING: the credit
     * grows with the distance up to ball_ref) */
    double db = sqrt((px - bx) * (px - bx) + (py - by) * (py - by));
    double ref = prm[PPS_ORACLE_R_BALL_REF];
    double x_ball = (db < ref ? db : ref) / ref;
    /* 3. angle to the goal: the best chance lies in a range of angles off
     * the goal axis, not at 0 (READING: full credit in [lo, hi], falling
     * linearly to 0 over span on either side) */
    double alpha = fabs(atan2(gy, gx));
    double lo = prm[PPS_ORACLE_R_ANGLE_LO], hi = prm[PPS_ORACLE_R_ANGLE_HI];
    double off = alpha < lo ? lo - alpha : (alpha > hi ? alpha - hi : 0.0);
    double f = off / prm[PPS_ORACLE_R_ANGLE_SPAN];
    double x_angle = 1.0 - (f > 1.0 ? 1.0 : f);
    /* 4. the opponent guards' time: P and Q are where the lines from p to
     * the two goal posts enter the defence area; the guards are the
     * opponents inside it (READING: the time to each of P and Q is the
     * fastest guard's, capped; no guard or no entry scores the cap) */
    double cap = prm[PPS_ORACLE_R_GUARD_CAP];
    double tsum = 0.0;
    for (int side = 0; side < 2; ++side) {
        double ex, ey, T = cap;
        if (segment_entry(px, py, x1, side ? hw : -hw, x0, x1, y0, y1, &ex,
                          &ey)) {
            for (int j = 0; j < st->n_opp; ++j) {
                const double* o = st->opp + 4 * j;
                if (o[0] < x0 || o[0] > x1 || o[1] < y0 || o[1] > y1) continue;
                double t = pps_oracle_intercept_time(o[0], o[1], o[2], o[3], ex,
                                                     ey, vmax, amax, 0.0);
                if (t < T) T = t;
            }
        }
        tsum += T;
    }
    double x_guard = tsum / (2.0 * cap);
    /* 5. avoid the opponent's defence: a cost when some opponent is nearer
     * the ball than p, so it would reach the ball first */
    double x_avoid = 0.0;
    for (int j = 0; j < st->n_opp; ++j) {
        const double* o = st->opp + 4 * j;
        double dj = sqrt((o[0] - bx) * (o[0] - bx) + (o[1] - by) * (o[1] - by));
        if (dj < db) x_avoid = 1.0;
    }
    /* READING: attackers may not stand inside the opponent's defence area,
     * so its interior holds no candidate; its edge (within the tolerance)
     * does */
    double tol = edge_tol(prm);
    int cand = !(px > x0 + tol && py > y0 + tol && py < y1 - tol);
    out[0] = cand ? -prm[PPS_ORACLE_R_W_GOAL] * x_goal
                        + prm[PPS_ORACLE_R_W_BALL] * x_ball
                        + prm[PPS_ORACLE_R_W_ANGLE] * x_angle
                        + prm[PPS_ORACLE_R_W_GUARD] * x_guard
                        - prm[PPS_ORACLE_R_W_AVOID] * x_avoid
                  : -INFINITY;
    out[1] = zone_of(st, px, py, tol);
    out[2] = x_goal;
    out[3] = x_ball;
    out[4] = x_angle;
    out[5] = x_guard;
    out[6] = x_avoid;
    out[7] = cand;
}

void pps_oracle_run_choose(const int64_t* best_idx, const double* best_score,
                           int avoid, int n_run, int* chosen)
{
    int k = 0;
    for (int z = 0; z < 4; ++z) chosen[z] = -1;
    /* the front pair (III, IV) first, then I, II */
    for (int pair = 1; pair >= 0; --pair) {
        int a = 2 * pair, b = 2 * pair + 1;
        int first = best_score[b] > best_score[a] ? b : a;
        int order[2] = {first, first == a ? b : a};
        for (int t = 0; t < 2; ++t) {
            int z = order[t];
            if (k < n_run && best_idx[z] >= 0 && z != avoid) chosen[k++] = z;
        }
    }
}

int pps_oracle_run_search(int S, const double* sc, const int* n_opp,
                          const double* opp, int jstride, const double* prm,
                          const double* pass, int64_t* best_idx,
                          double* best_score, int* chosen, int* avoided,
                          double* score, int n_threads)
{
    double g = prm[PPS_ORACLE_R_SPACING];
    if (S < 0 || !(g > 0.0)) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int s = 0; s < S; ++s) {
        pps_oracle_dpps_state st;
        st.sc = sc + (int64_t)s * PPS_ORACLE_NSCALAR;
        st.n_team = 0;
        st.team = NULL;
        st.n_opp = n_opp[s];
        st.opp = opp + (int64_t)s * jstride * 4;
        st.K = 1;
        double L = st.sc[PPS_ORACLE_FIELD_LEN], W = st.sc[PPS_ORACLE_FIELD_WID];
        int nx = (int)lround(0.5 * L / g) + 1, ny = (int)lround(W / g) + 1;
        int64_t* bi = best_idx + 4 * s;
        double* bs = best_score + 4 * s;
        for (int z = 0; z < 4; ++z) {
            bi[z] = -1;
            bs[z] = -INFINITY;
        }
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double out[8];
                /* READING: the raster spans the attacking half exactly;
                 * its last column lies on the goal line and its last row
                 * on the touch line, whatever the rounding of i g */
                double px = fmin(i * g, 0.5 * L);
                double py = fmin(-0.5 * W + j * g, 0.5 * W);
                pps_oracle_run_point(&st, prm, px, py, out);
                int64_t idx = (int64_t)j * nx + i;
                int z = (int)out[1];
                if (score) score[(int64_t)s * nx * ny + idx] = out[0];
                if (out[7] != 0.0 && (bi[z] < 0 || out[0] > bs[z])) {
                    bi[z] = idx;
                    bs[z] = out[0];
                }
            }
        int av = -1;
        if (pass && !isnan(pass[2 * s]) && !isnan(pass[2 * s + 1]))
            av = pps_oracle_run_zone(&st, prm, pass[2 * s], pass[2 * s + 1]);
        avoided[s] = av;
        pps_oracle_run_choose(bi, bs, av, (int)prm[PPS_ORACLE_R_N_RUN],
                              chosen + 4 * s);
    }
    (void)n_threads;
    return 0;
}

int pps_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
