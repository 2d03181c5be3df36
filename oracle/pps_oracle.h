/*
 * pps_oracle.h -- plain FP64 CPU oracle for the passing-point search of the
 * ZJUNlict 2019 team description paper (Sec. 4.1 ball model, Sec. 4.2
 * SBIP-based dynamic passing-point search, Sec. 4.3 value-based best pass,
 * Sec. 4.4 shooting, Sec. 5.1-5.2 running points).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path; it defines its own state
 * layout (plain double arrays) and its own grid rule.
 *
 * The paper describes the method in prose only.  Where it is silent this
 * oracle takes a stated reading, marked READING in pps_oracle.c.
 *
 * Parity pins (checked by the CPU test suite against closed forms, brute
 * force time stepping and invariants): ball time, intercept time, margin,
 * shot angle, score, argmax tie rule, grid counts.  No function here is
 * "parity unpinned".
 */
#ifndef PPS_ORACLE_H
#define PPS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Per-state scalar record, 8 doubles, in this order. */
enum {
    PPS_ORACLE_BALL_X = 0,
    PPS_ORACLE_BALL_Y = 1,
    PPS_ORACLE_BALL_DECEL = 2, /* rolling deceleration a (m/s^2), > 0 */
    PPS_ORACLE_VMAX = 3,       /* opponent speed limit (m/s) */
    PPS_ORACLE_AMAX = 4,       /* opponent acceleration limit (m/s^2) */
    PPS_ORACLE_FIELD_LEN = 5,  /* L, along x; opponent goal at x = +L/2 */
    PPS_ORACLE_FIELD_WID = 6,  /* W, along y */
    PPS_ORACLE_GOAL_WIDTH = 7, /* goal mouth width */
    PPS_ORACLE_NSCALAR = 8
};

/* Value-function and feasibility parameters, 8 doubles, in this order. */
enum {
    PPS_ORACLE_W_ANGLE = 0,
    PPS_ORACLE_W_DIST = 1,
    PPS_ORACLE_W_MARGIN = 2,
    PPS_ORACLE_MARGIN_CAP = 3,
    PPS_ORACLE_TAU_SAFE = 4,
    PPS_ORACLE_ROBOT_RADIUS = 5, /* disc radius for shot blocking */
    PPS_ORACLE_REACH_RADIUS = 6, /* intercept reach radius */
    PPS_ORACLE_MIN_PASS_DIST = 7,
    PPS_ORACLE_NPARAM = 8
};

/* One state as the oracle sees it: scalars (8 doubles), n_opp opponents
 * (x, y, vx, vy each) and the sample count K. */
typedef struct {
    const double* sc;  /* PPS_ORACLE_NSCALAR values */
    int n_opp;
    const double* opp; /* n_opp x 4 */
    int K;
} pps_oracle_state;

/* Grid rule: x0 = -L/2, y0 = -W/2, nx = round(L/g)+1, ny = round(W/g)+1. */
void pps_oracle_grid(double L, double W, double g, int* nx, int* ny,
                     double* x0, double* y0);

/* Ball arrival time at distance s for kick speed v, deceleration a
 * (+inf beyond the stopping distance). */
double pps_oracle_ball_time(double s, double v, double a);

/* Minimum time for an opponent at (ox, oy) with velocity (ux, uy) to bring
 * its centre within reach of (px, py). */
double pps_oracle_intercept_time(double ox, double oy, double ux, double uy,
                                 double px, double py, double vmax,
                                 double amax, double reach);

/* Minimum over opponents of the intercept time of point (px, py);
 * +inf without opponents. */
double pps_oracle_min_intercept(const pps_oracle_state* st, double px,
                                double py, double reach);

/* pps_oracle_min_intercept at n points pxy[2i], pxy[2i+1] -> out[i]. */
void pps_oracle_min_intercept_many(const pps_oracle_state* st, int n,
                                   const double* pxy, double reach,
                                   double* out);

/* Safety margin of the pass to (cx, cy) at kick speed v:
 * min_k (T_k - t_ball(s_k)), k = 1..K.  Writes T_k to T_out[k-1] when
 * T_out is not NULL, and the reachability to *reachable.  -inf when the
 * ball stops short of the receiver. */
double pps_oracle_margin(const pps_oracle_state* st, double cx, double cy,
                         double v, double reach, double* T_out,
                         int* reachable);

/* Largest unblocked angular gap of the opponent goal mouth seen from
 * (cx, cy), opponents as discs of radius r. */
double pps_oracle_shot_angle(const pps_oracle_state* st, double cx,
                             double cy, double r);

/* Score of a feasible candidate (Eq. 3 with the three features of the
 * build: shot angle, goal distance, margin). */
double pps_oracle_score(const pps_oracle_state* st, const double* prm,
                        double cx, double cy, double margin);

/* Full search over a batch of states sharing one grid and speed list.
 *
 * sc:     S x 8 scalars; n_opp: S; K: S; opp: S x jstride x 4.
 * Grid point (ix, iy) = (x0 + ix*g, y0 + iy*g); P = nx*ny, p = iy*nx + ix.
 * Candidate index idx = v*P + p.
 * Outputs per state: best_idx (-1 if none), best_score (-inf if none),
 * best_margin, n_feasible.  Optional (NULL to skip): feasible[S][V][P],
 * margin[S][V][P], score[S][V][P] (-inf when infeasible), T[S][P][kstride]
 * (intercept times along the first speed's pass line).
 * n_threads <= 0 uses the OpenMP default.  Returns 0, or -1 on bad input. */
int pps_oracle_search(int S, const double* sc, const int* n_opp,
                      const int* K, int jstride, const double* opp,
                      double g, int nx, int ny, double x0, double y0,
                      const double* speeds, int V, const double* prm,
                      int64_t* best_idx, double* best_score,
                      double* best_margin, int64_t* n_feasible,
                      uint8_t* feasible, double* margin, double* score,
                      double* T, int kstride, int n_threads);

/* Threads the OpenMP runtime will use (1 without OpenMP). */
/* ---- D: the paper's own search, directions x kick powers (Sec. 4.2) ----
 *
 * From the ball holder at b, candidate passes are ndir directions
 * (phi_i = 2 pi i / ndir) x npow kick powers (v0_j uniform in [vlo, vhi]);
 * for every candidate the ball's path is searched for the first teammate
 * and the first opponent interception (SBIP), and feasible candidates are
 * scored with the features of Sec. 4.3.  Parameters, 13 doubles: */
enum {
    PPS_ORACLE_D_VLO = 0,        /* lowest kick power (m/s) */
    PPS_ORACLE_D_VHI = 1,        /* highest kick power */
    PPS_ORACLE_D_SLIDE = 2,      /* rolling speed / kick speed (5/7) */
    PPS_ORACLE_D_TAU_DELTA = 3,  /* feasible iff t_opp - t_team > this */
    PPS_ORACLE_D_DELTA_CAP = 4,  /* cap of the delta-time feature (s) */
    PPS_ORACLE_D_W_TIME = 5,     /* weight of -t_team */
    PPS_ORACLE_D_W_ANGLE = 6,    /* weight of the shot angle / pi */
    PPS_ORACLE_D_W_DIST = 7,     /* weight of -|g - p| / diag */
    PPS_ORACLE_D_W_REFR = 8,     /* weight of -refraction angle / pi */
    PPS_ORACLE_D_W_DELTA = 9,    /* weight of min(t_opp - t_team, cap) */
    PPS_ORACLE_D_ROBOT_RADIUS = 10,
    PPS_ORACLE_D_REACH_RADIUS = 11,
    PPS_ORACLE_D_MIN_TIME = 12,  /* reserved, 0 */
    PPS_ORACLE_D_NPARAM = 13
};

/* A state of the direction x power search: scalars as above (the ball is
 * at the passer's feet), n_team receivers and n_opp opponents (x, y, vx,
 * vy each), K samples along each ball path. */
typedef struct {
    const double* sc;
    int n_team;
    const double* team; /* n_team x 4 */
    int n_opp;
    const double* opp;  /* n_opp x 4 */
    int K;
} pps_oracle_dpps_state;

/* Length of the ball's path from b along direction (ux, uy) at rolling
 * speed v: the stopping distance, or the distance to the field edge if
 * that comes first (*stopped = 0 then). */
double pps_oracle_dpps_path(const pps_oracle_dpps_state* st, double ux,
                            double uy, double v, int* stopped);

/* First interception of the ball's path by one group of robots (n x 4):
 * the first sample k = 1..K whose ball time t_k is not earlier than the
 * group's minimum intercept time there; at the stop sample of a path that
 * ends by stopping, the group always gets the ball, at max(T, t_K).
 * Returns the time (+inf if none); *k_out = k (0 if none); *who = the
 * robot with the minimum intercept time at that sample. */
double pps_oracle_dpps_group(const pps_oracle_dpps_state* st, int n,
                             const double* robots, double ux, double uy,
                             double v, double reach, int* k_out, int* who);

/* The same, also giving the smallest |T - t_ball| over the samples it
 * searched before deciding (+inf if none): how far the decision was from
 * flipping. */
double pps_oracle_dpps_group_margin(const pps_oracle_dpps_state* st, int n,
                                    const double* robots, double ux,
                                    double uy, double v, double reach,
                                    int* k_out, int* who, double* margin);

/* One candidate (direction i of ndir, power j of npow): out[0] t_team,
 * out[1] t_opp, out[2] k_team, out[3] receiver, out[4] receive x,
 * out[5] receive y, out[6] feasible (0/1), out[7] score (-inf if not),
 * out[8] / out[9] the teammate / opponent decision margins. */
void pps_oracle_dpps_candidate(const pps_oracle_dpps_state* st,
                               const double* prm, int ndir, int npow, int i,
                               int j, double* out);

/* The search over S states: state s has scalars sc + 8 s, n_team[s]
 * receivers at team + 4 jstride s, n_opp[s] opponents at opp + 4 jstride s,
 * K[s] samples.  Best idx = i * npow + j (-1 if none; equal scores go to
 * the smaller idx), its score and the feasible count; optional dense
 * outputs of S x ndir x npow: feasible, score, t_team, t_opp.  Returns 0,
 * or -1 on bad arguments. */
int pps_oracle_dpps_search(int S, const double* sc, const int* n_team,
                           const double* team, const int* n_opp,
                           const double* opp, const int* K, int jstride,
                           int ndir, int npow, const double* prm,
                           int64_t* best_idx, double* best_score,
                           int64_t* n_feasible, uint8_t* feasible,
                           double* score, double* t_team, double* t_opp,
                           int n_threads);

/* Passing power (Sec. 4.1, Eq. 1-2) for receiver `receiver` of st and the
 * target (tx, ty): out[0] kick power v0, out[1] rolling speed v1, out[2]
 * pass time t = T + buffer, out[3] the receiver's arrival T (C3), out[4]
 * clamped to [v_lo, v_hi] (0/1). */
void pps_oracle_pass_power(const pps_oracle_dpps_state* st, int receiver,
                           double tx, double ty, double buffer, double slide,
                           double v_lo, double v_hi, double reach,
                           double* out);

/* Shooting decision (Sec. 4.4) from (cx, cy): out[0] the open angle,
 * out[1] the shot direction (middle of the largest gap), out[2] the ball's
 * time to the goal line (+inf if it stops short), out[3] the first
 * opponent's interception time along the shot (+inf if none), out[4]
 * shoot (0/1), out[5] the smallest |T - t_ball| over the samples searched
 * (how far the interception decision was from flipping). */
void pps_oracle_shoot(const pps_oracle_dpps_state* st, double cx, double cy,
                      double v_shot, double slide, double theta_min,
                      double tau, double robot_radius, double reach,
                      double* out);

/* The shot angle (C6) and where its gap starts (*start, radians). */
double pps_oracle_shot_gap(const pps_oracle_state* st, double cx, double cy,
                           double r, double* start);

/* ---- R: running points (Sec. 5.1-5.2) ----
 * The attacking half is rasterised (x = min(i g, L/2), i = 0..round(L/2/g);
 * y = min(-W/2 + j g, W/2), j = 0..round(W/g)) and split into four zones: I, II
 * behind x = L/4, III, IV in front of it, each pair split at the ball's y
 * (kept within +-W/4, so the zones move with the ball).  A point within
 * spacing / 1024 of a cut or of the defence area's edge counts as on it.
 * Every grid point outside the opponent's defence area (its edge included)
 * is scored by the weighted sum of the
 * five criteria of Sec. 5.2 (Eq. 4); the best point of each zone is the
 * zone's running point.  Parameters, PPS_ORACLE_R_NPARAM doubles: */
enum {
    PPS_ORACLE_R_SPACING = 0,
    PPS_ORACLE_R_W_GOAL = 1,     /* weight of |goal - p| / diagonal (a cost) */
    PPS_ORACLE_R_W_BALL = 2,     /* weight of min(|p - b|, ball_ref) / ball_ref */
    PPS_ORACLE_R_W_ANGLE = 3,    /* weight of the angle-to-goal credit */
    PPS_ORACLE_R_W_GUARD = 4,    /* weight of the guards' time to P and Q */
    PPS_ORACLE_R_W_AVOID = 5,    /* weight of the defence-avoidance cost */
    PPS_ORACLE_R_BALL_REF = 6,   /* m */
    PPS_ORACLE_R_ANGLE_LO = 7,   /* rad: full credit for angles in [lo, hi] */
    PPS_ORACLE_R_ANGLE_HI = 8,
    PPS_ORACLE_R_ANGLE_SPAN = 9, /* rad: the credit falls to 0 over this span */
    PPS_ORACLE_R_DEF_DEPTH = 10, /* defence area depth (m) */
    PPS_ORACLE_R_DEF_WIDTH = 11, /* defence area width (m) */
    PPS_ORACLE_R_GUARD_CAP = 12, /* s: cap of each guard time */
    PPS_ORACLE_R_N_RUN = 13,     /* supporters to place, 0..4 */
    PPS_ORACLE_R_NPARAM = 14
};

/* The point (px, py) of state st (its ball and opponents; teammates
 * unused): out[0] score (-inf inside the defence area), out[1] zone 0..3
 * (I..IV), out[2..6] the criteria (goal distance, ball, angle, guard,
 * avoid), out[7] 1 if a candidate (outside the defence area). */
void pps_oracle_run_point(const pps_oracle_dpps_state* st, const double* prm,
                          double px, double py, double* out);

/* Zone of a point of the attacking half (-1 outside it); the cuts take the
 * edge tolerance spacing / 1024 of prm. */
int pps_oracle_run_zone(const pps_oracle_dpps_state* st, const double* prm,
                        double px, double py);

/* Sec. 5.1's choice of zones for n_run supporters: zones without a point
 * and the zone `avoid` (the best passing point's, -1 none) are left out;
 * zones III and IV come before I and II, each pair by score (the lower
 * zone first on ties).  chosen[0..3]: zones in that order, -1 after the
 * last. */
void pps_oracle_run_choose(const int64_t* best_idx, const double* best_score,
                           int avoid, int n_run, int* chosen);

/* All states: per state and zone the best grid index j * nx + i (-1 if the
 * zone holds no candidate; the lowest index on ties) and score, the chosen
 * zones and the avoided zone.  pass: S x 2 best passing points (NaN: none)
 * or NULL.  score: optional dense scores, S x ny x nx. */
int pps_oracle_run_search(int S, const double* sc, const int* n_opp,
                          const double* opp, int jstride, const double* prm,
                          const double* pass, int64_t* best_idx,
                          double* best_score, int* chosen, int* avoided,
                          double* score, int n_threads);

int pps_oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
