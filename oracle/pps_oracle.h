/*
 * pps_oracle.h -- plain FP64 CPU oracle for the passing-point search of the
 * ZJUNlict 2019 team description paper (Sec. 4.1 ball model, Sec. 4.2
 * SBIP-based dynamic passing-point search, Sec. 4.3 value-based best pass).
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
int pps_oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
