// pps_cells.cuh -- the cell lattice shared by the proposal network's map
// and the fine grids it ranks (labels, top-k, refinement).
#pragma once

#include <math.h>

#include "pps.h"

namespace pps {
namespace net {

constexpr int kMapH = PPS_NET_H, kMapW = PPS_NET_W;

// ------------------------------------------------------------ cell lattice
// Map pixel (cx, cy) is centred at (-6 + 0.2 cx, -4.5 + 0.2 cy).  A fine
// grid of spacing g = 0.2 / m (m = 1, 2, 4 or 8) whose points fall on the
// same lattice gives each pixel the m x m points nearest its centre: fine
// columns m cx + ox .. m cx + ox + m - 1 and rows m cy + oy .. + m - 1,
// with ox = (-6 - x0) / g - m / 2 and oy = (-4.5 - y0) / g - m / 2 (the
// 0.025 m grid of the 12 x 9 m field: 8 cx - 4 .. 8 cx + 3).  Every fine
// point belongs to exactly one cell.
struct CellLattice {
    int m, ox, oy;
    bool ok;
};

__host__ __device__ inline CellLattice cell_lattice(const pps_grid& g) {
    CellLattice c{0, 0, 0, false};
    if (!(g.spacing > 0.f) || g.nx < 1 || g.ny < 1) return c;
    const float mf = 0.2f / g.spacing;
    const int m = (int)(mf + 0.5f);
    if (!(m == 1 || m == 2 || m == 4 || m == 8) ||
        fabsf(mf - (float)m) > 1e-4f * (float)m)
        return c;
    const float fx = (-6.f - g.x0) / g.spacing, fy = (-4.5f - g.y0) / g.spacing;
    const float rx = floorf(fx + 0.5f), ry = floorf(fy + 0.5f);
    if (fabsf(fx - rx) > 1e-3f || fabsf(fy - ry) > 1e-3f) return c;
    c.m = m;
    c.ox = (int)rx - m / 2;
    c.oy = (int)ry - m / 2;
    // the grid must lie inside the map's 46 x 61 cells
    c.ok = c.ox <= 0 && c.oy <= 0 && (g.nx - 1 - c.ox) / m < kMapW &&
           (g.ny - 1 - c.oy) / m < kMapH;
    return c;
}

// Does the cell of map pixel (cx, cy) hold any point of the grid?
__host__ __device__ inline bool cell_on_grid(const CellLattice& c,
                                             const pps_grid& g, int cx,
                                             int cy) {
    const int x0 = c.m * cx + c.ox, y0 = c.m * cy + c.oy;
    return x0 + c.m > 0 && x0 < g.nx && y0 + c.m > 0 && y0 < g.ny;
}

}  // namespace net
}  // namespace pps
