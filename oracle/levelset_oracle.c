/*
 * levelset_oracle.c -- plain, slow, FP64 CPU oracle of the narrow-band
 * first-order upwind level-set step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or constant with the CUDA
 * library.
 *
 * Paper: Z. Wang, "Parallel Level set algorithm with MPI and accelerated on
 * GPU" (arXiv 1612.04040).  Equations are numbered in order of appearance:
 *   Eq. 1  phi(x,0) = +-d                                  (section 1)
 *   Eq. 2  phi_t + F|grad phi| = 0                         (section 1)
 *   Eq. 3  phi^{n+1} = phi^n - dt[max(F,0) G+ + min(F,0) G-] (section 1)
 *   Eq. 4  G+ = sqrt(sum over axes of max(D-,0)^2 + min(D+,0)^2)
 *   Eq. 5  G- = sqrt(sum over axes of max(D+,0)^2 + min(D-,0)^2)
 *   Eq. 6  tube T = {x : |phi(x)| < gamma}                (section 1.1)
 *   Eq. 7  cut-off c(|phi|): 1 up to beta, cubic to 0 at gamma (section 1.1)
 *   Eq. 8  phi_t + c(phi) F |grad phi| = 0 on T           (section 1.1)
 *   Eq. 10 clamp of the reinitialised d to [-gamma, gamma] (section 1.1)
 *   Eq. 11 region N = points with a +-dx neighbour in T    (section 1.1)
 *   Eq. 12 d_tau + S(d)(|grad d| - 1) = 0, d(x,0) = phi-bar (section 1.1)
 *   Eq. 13 S = d / sqrt(d^2 + |Dd|^2 dx^2)                 (section 1.1)
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - D-x = (phi_i - phi_{i-1})/h, D+x = (phi_{i+1} - phi_i)/h, and the same
 *     for y and z (textbook one-sided differences of the scheme the paper
 *     cites for Eq. 3-5).
 *   - The six squared terms of Eq. 4/5 are summed per axis first,
 *     s_a = max(..)^2 + min(..)^2, then ((s_x + s_y) + s_z).
 *   - Domain faces: a missing one-sided difference equals the existing one on
 *     the same axis ("extrapolate", the default), or is 0 ("neumann": ghost
 *     value equal to the edge value).
 *   - Band granularity: the tube test of Eq. 6 is applied per tile of
 *     tile^3 points (a tile is "core" when one of its points is in T); the
 *     active set is the core set dilated by one tile (26 or 6 neighbours).
 *     tile = 1 with the 6-neighbour dilation gives exactly the pointwise T
 *     and N of Eq. 6 and Eq. 11.  Points outside active tiles do not change.
 *
 *   - Local scheme (Steps 1-3 of section 1.1): Eq. 8 is discretised as
 *     Eq. 3 with the speed c(|phi^n|) F; N (Eq. 11) is the point set whose
 *     point or one of its six face neighbours is in T, taken from phi^n;
 *     Eq. 12 is iterated a given number of times with the upwind gradient of
 *     Eq. 4 where d > 0 and of Eq. 5 where d < 0 (S carries the sign of d),
 *     |Dd| in Eq. 13 is that same gradient, the pseudo time step is a given
 *     dtau; then Eq. 10 clamps the values on N.  Points outside N keep
 *     their value throughout.
 *
 * Layout: phi[z][y][x], x fastest: index = (z*ny + y)*nx + x.
 * Build: -O2 -ffp-contract=off (no fused multiply-add anywhere), optional
 * OpenMP over z planes; every result is independent of the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BC_EXTRAPOLATE 0
#define ORC_BC_NEUMANN 1

static size_t idx3(int nx, int ny, int x, int y, int z)
{
    return ((size_t)z * (size_t)ny + (size_t)y) * (size_t)nx + (size_t)x;
}

static double max0(double a) { return a > 0.0 ? a : 0.0; }
static double min0(double a) { return a < 0.0 ? a : 0.0; }

/* One-sided differences D-, D+ of phi at position pos along one axis of
 * length n, stride `stride` in the flat array (Eq. 4/5 symbols). */
static void one_sided(const double *phi, size_t i, size_t stride, int pos, int n,
                      double h, int bc, double *dm, double *dp)
{
    const double c = phi[i];
    const int has_m = pos > 0;
    const int has_p = pos < n - 1;
    double m = 0.0, p = 0.0;
    if (has_m) m = (c - phi[i - stride]) / h;
    if (has_p) p = (phi[i + stride] - c) / h;
    if (bc == ORC_BC_EXTRAPOLATE) {
        if (!has_m && has_p) m = p;
        if (!has_p && has_m) p = m;
    }
    /* neumann: the ghost value equals the edge value, so the missing
     * difference stays 0 */
    *dm = m;
    *dp = p;
}

/* Eq. 3-5 at one grid point.  Returns phi^{n+1} at (x, y, z). */
double orc_point_update(int nx, int ny, int nz, double h, int bc,
                        const double *phi, double F, double dt,
                        int x, int y, int z)
{
    const size_t i = idx3(nx, ny, x, y, z);
    double dmx, dpx, dmy, dpy, dmz, dpz;
    one_sided(phi, i, 1, x, nx, h, bc, &dmx, &dpx);
    one_sided(phi, i, (size_t)nx, y, ny, h, bc, &dmy, &dpy);
    one_sided(phi, i, (size_t)nx * (size_t)ny, z, nz, h, bc, &dmz, &dpz);

    /* Eq. 4: max(D-,0)^2 + min(D+,0)^2 per axis */
    const double ax = max0(dmx), bx = min0(dpx);
    const double ay = max0(dmy), by = min0(dpy);
    const double az = max0(dmz), bz = min0(dpz);
    const double spx = ax * ax + bx * bx;
    const double spy = ay * ay + by * by;
    const double spz = az * az + bz * bz;
    const double gplus = sqrt((spx + spy) + spz);

    /* Eq. 5: max(D+,0)^2 + min(D-,0)^2 per axis */
    const double cx = max0(dpx), ex = min0(dmx);
    const double cy = max0(dpy), ey = min0(dmy);
    const double cz = max0(dpz), ez = min0(dmz);
    const double smx = cx * cx + ex * ex;
    const double smy = cy * cy + ey * ey;
    const double smz = cz * cz + ez * ez;
    const double gminus = sqrt((smx + smy) + smz);

    /* Eq. 3 */
    return phi[i] - dt * (max0(F) * gplus + min0(F) * gminus);
}

static size_t tile_of(int tile, int tnx, int tny, int x, int y, int z)
{
    return ((size_t)(z / tile) * (size_t)tny + (size_t)(y / tile)) * (size_t)tnx
           + (size_t)(x / tile);
}

/* One upwind step (Eq. 3) on every point of every active tile; points of
 * inactive tiles are copied unchanged.  tile_active == NULL: whole domain.
 * F == NULL: constant speed Fc. */
void orc_step(int nx, int ny, int nz, double h, int bc, const double *phi,
              const double *F, double Fc, const uint8_t *tile_active, int tile,
              double dt, double *out)
{
    const int tnx = (nx + tile - 1) / tile;
    const int tny = (ny + tile - 1) / tile;
    int z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; ++z) {
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                const size_t i = idx3(nx, ny, x, y, z);
                if (tile_active && !tile_active[tile_of(tile, tnx, tny, x, y, z)]) {
                    out[i] = phi[i];
                    continue;
                }
                const double f = F ? F[i] : Fc;
                out[i] = orc_point_update(nx, ny, nz, h, bc, phi, f, dt, x, y, z);
            }
        }
    }
}

/* Eq. 3 at a list of points (flat indices), reading phi only: for sampled
 * checks of large grids. */
void orc_step_points(int nx, int ny, int nz, double h, int bc, const double *phi,
                     const double *Fpts, double dt, const int64_t *pts, int64_t npts,
                     double *out)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < npts; ++k) {
        const int64_t i = pts[k];
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((int64_t)nx * ny));
        out[k] = orc_point_update(nx, ny, nz, h, bc, phi, Fpts[k], dt, x, y, z);
    }
}

/* Eq. 6 per tile: core[t] = 1 when some point p of tile t has |phi_p| < gamma
 * (strict). */
void orc_classify(int nx, int ny, int nz, int tile, const double *phi,
                  double gamma, uint8_t *core)
{
    const int tnx = (nx + tile - 1) / tile;
    const int tny = (ny + tile - 1) / tile;
    const int tnz = (nz + tile - 1) / tile;
    const size_t ntiles = (size_t)tnx * tny * tnz;
    memset(core, 0, ntiles);
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                if (fabs(phi[idx3(nx, ny, x, y, z)]) < gamma)
                    core[tile_of(tile, tnx, tny, x, y, z)] = 1;
}

/* Band dilation: active = core plus every tile sharing a face (conn = 6) or
 * a face, edge or corner (conn = 26) with a core tile. */
void orc_dilate(int tnx, int tny, int tnz, const uint8_t *core, int conn,
                uint8_t *active)
{
    for (int z = 0; z < tnz; ++z)
        for (int y = 0; y < tny; ++y)
            for (int x = 0; x < tnx; ++x) {
                int on = 0;
                for (int dz = -1; dz <= 1 && !on; ++dz)
                    for (int dy = -1; dy <= 1 && !on; ++dy)
                        for (int dx = -1; dx <= 1 && !on; ++dx) {
                            const int manhattan = abs(dx) + abs(dy) + abs(dz);
                            if (conn == 6 && manhattan > 1) continue;
                            const int X = x + dx, Y = y + dy, Z = z + dz;
                            if (X < 0 || Y < 0 || Z < 0 || X >= tnx || Y >= tny || Z >= tnz)
                                continue;
                            if (core[((size_t)Z * tny + Y) * tnx + X]) on = 1;
                        }
                active[((size_t)z * tny + y) * tnx + x] = (uint8_t)on;
            }
}

/* Active-point array (section 2): ascending ids of the set flags. */
int64_t orc_compact(const uint8_t *flags, int64_t n, int32_t *ids)
{
    int64_t k = 0;
    for (int64_t t = 0; t < n; ++t)
        if (flags[t]) ids[k++] = (int32_t)t;
    return k;
}

/* CFL speed bound: max |F| over the points of active tiles (all points when
 * tile_active == NULL).  0 when there is no such point. */
double orc_max_abs_speed(int nx, int ny, int nz, int tile, const double *F,
                         double Fc, const uint8_t *tile_active)
{
    const int tnx = (nx + tile - 1) / tile;
    const int tny = (ny + tile - 1) / tile;
    double m = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (tile_active && !tile_active[tile_of(tile, tnx, tny, x, y, z)])
                    continue;
                const double a = fabs(F ? F[idx3(nx, ny, x, y, z)] : Fc);
                if (a > m) m = a;
            }
    return m;
}

/* ------------------------------------------------------------------------
 * Learned coarse-grid corrector (not in the paper): plain FP64 building
 * blocks, written from their definitions.
 *
 * Layout: activations channels-last x[(z*ny + y)*nx + x][c]; weights
 * W[tap][ci][co] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1), dx, dy, dz in
 * {-1, 0, 1}; zero padding outside the grid.
 * ---------------------------------------------------------------------- */

/* y[p][o] = b[o] + sum_tap sum_ci x[p + off(tap)][ci] * W[tap][ci][o] */
void orc_conv3_fwd(int nx, int ny, int nz, int ci, int co, const double *x, const double *W,
                   const double *b, double *y)
{
    int z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy)
            for (int xx = 0; xx < nx; ++xx) {
                double *out = y + idx3(nx, ny, xx, yy, z) * (size_t)co;
                for (int o = 0; o < co; ++o) out[o] = b ? b[o] : 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int X = xx + dx, Y = yy + dy, Z = z + dz;
                            if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                            const int tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                            const double *in = x + idx3(nx, ny, X, Y, Z) * (size_t)ci;
                            const double *w = W + (size_t)tap * ci * co;
                            for (int c = 0; c < ci; ++c)
                                for (int o = 0; o < co; ++o) out[o] += in[c] * w[c * co + o];
                        }
            }
}

/* dx[q][ci] = sum_tap sum_o dy[q - off(tap)][o] * W[tap][ci][o]  (the adjoint
 * of orc_conv3_fwd with respect to x) */
void orc_conv3_bwd_data(int nx, int ny, int nz, int ci, int co, const double *dy,
                        const double *W, double *dxo)
{
    int z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; ++z)
        for (int yy = 0; yy < ny; ++yy)
            for (int xx = 0; xx < nx; ++xx) {
                double *out = dxo + idx3(nx, ny, xx, yy, z) * (size_t)ci;
                for (int c = 0; c < ci; ++c) out[c] = 0.0;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dyy = -1; dyy <= 1; ++dyy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            /* output point p with p + off(tap) = q */
                            const int X = xx - dx, Y = yy - dyy, Z = z - dz;
                            if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                            const int tap = (dz + 1) * 9 + (dyy + 1) * 3 + (dx + 1);
                            const double *g = dy + idx3(nx, ny, X, Y, Z) * (size_t)co;
                            const double *w = W + (size_t)tap * ci * co;
                            for (int c = 0; c < ci; ++c)
                                for (int o = 0; o < co; ++o) out[c] += g[o] * w[c * co + o];
                        }
            }
}

/* dW[tap][ci][o] = sum_p x[p + off(tap)][ci] * dy[p][o];  db[o] = sum_p dy[p][o].
 * Each tap's sums run over the points in ascending order; the taps are
 * independent (one OpenMP task each), so the result does not depend on the
 * thread count. */
void orc_conv3_bwd_weight(int nx, int ny, int nz, int ci, int co, const double *x,
                          const double *dy, double *dW, double *db)
{
    int tap;
    memset(dW, 0, sizeof(double) * 27 * (size_t)ci * co);
    if (db) {
        memset(db, 0, sizeof(double) * (size_t)co);
        for (size_t p = 0; p < (size_t)nx * ny * nz; ++p)
            for (int o = 0; o < co; ++o) db[o] += dy[p * (size_t)co + o];
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (tap = 0; tap < 27; ++tap) {
        const int dx = tap % 3 - 1, dyy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
        double *w = dW + (size_t)tap * ci * co;
        for (int z = 0; z < nz; ++z)
            for (int yy = 0; yy < ny; ++yy)
                for (int xx = 0; xx < nx; ++xx) {
                    const int X = xx + dx, Y = yy + dyy, Z = z + dz;
                    if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                    const double *g = dy + idx3(nx, ny, xx, yy, z) * (size_t)co;
                    const double *in = x + idx3(nx, ny, X, Y, Z) * (size_t)ci;
                    for (int c = 0; c < ci; ++c)
                        for (int o = 0; o < co; ++o) w[c * co + o] += in[c] * g[o];
                }
    }
}

/* restriction by 4: coarse value at the coarse cell centre (4I+2)h_f, i.e.
 * the trilinear value there = mean of the fine points 4I+1, 4I+2 per axis */
void orc_restrict4(int nfx, int nfy, int nfz, const double *fine, double *coarse)
{
    const int ncx = nfx / 4, ncy = nfy / 4, ncz = nfz / 4;
    for (int Z = 0; Z < ncz; ++Z)
        for (int Y = 0; Y < ncy; ++Y)
            for (int X = 0; X < ncx; ++X) {
                double s = 0.0;
                for (int k = 1; k <= 2; ++k)
                    for (int j = 1; j <= 2; ++j)
                        for (int i = 1; i <= 2; ++i)
                            s += fine[idx3(nfx, nfy, 4 * X + i, 4 * Y + j, 4 * Z + k)];
                coarse[idx3(ncx, ncy, X, Y, Z)] = s / 8.0;
            }
}

/* ------------------------------------------------------------------------
 * Local level-set scheme of section 1.1 (Steps 1-3): cut-off advance,
 * reinitialisation on N, clamp.
 * ---------------------------------------------------------------------- */

/* Eq. 7: the cut-off factor at a = |phi| for 0 < beta < gamma. */
double orc_cutoff(double a, double beta, double gamma)
{
    if (a <= beta) return 1.0;
    if (a < gamma) {
        const double u = a - gamma;
        const double w = gamma - beta;
        return (u * u) * ((2.0 * a + gamma) - 3.0 * beta) / ((w * w) * w);
    }
    return 0.0;
}

/* Eq. 8 discretised as Eq. 3 with the speed c(|phi^n|) F at every point
 * (c = 0 outside T, so those points keep their value). */
void orc_cut_step(int nx, int ny, int nz, double h, int bc, const double *phi,
                  const double *F, double Fc, double beta, double gamma, double dt,
                  double *out)
{
    int z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t i = idx3(nx, ny, x, y, z);
                const double f = F ? F[i] : Fc;
                const double c = orc_cutoff(fabs(phi[i]), beta, gamma);
                out[i] = orc_point_update(nx, ny, nz, h, bc, phi, f * c, dt, x, y, z);
            }
}

/* Eq. 11: nmask[i] = 1 when point i or one of its six face neighbours
 * (inside the domain) is in T, i.e. has |phi| < gamma. */
void orc_region_n(int nx, int ny, int nz, const double *phi, double gamma, uint8_t *nmask)
{
    int z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int in = fabs(phi[idx3(nx, ny, x, y, z)]) < gamma;
                if (!in && x > 0) in = fabs(phi[idx3(nx, ny, x - 1, y, z)]) < gamma;
                if (!in && x < nx - 1) in = fabs(phi[idx3(nx, ny, x + 1, y, z)]) < gamma;
                if (!in && y > 0) in = fabs(phi[idx3(nx, ny, x, y - 1, z)]) < gamma;
                if (!in && y < ny - 1) in = fabs(phi[idx3(nx, ny, x, y + 1, z)]) < gamma;
                if (!in && z > 0) in = fabs(phi[idx3(nx, ny, x, y, z - 1)]) < gamma;
                if (!in && z < nz - 1) in = fabs(phi[idx3(nx, ny, x, y, z + 1)]) < gamma;
                nmask[idx3(nx, ny, x, y, z)] = (uint8_t)in;
            }
}

/* One pseudo-time iteration of Eq. 12 at one point:
 *   g = G+ (Eq. 4) if d > 0, G- (Eq. 5) if d < 0;
 *   S = d / sqrt(d^2 + g^2 h^2)                      (Eq. 13, |Dd| = g)
 *   d_new = d - dtau * (S * (g - 1)).
 * d = 0 gives S = 0: the value stays. */
double orc_reinit_point(int nx, int ny, int nz, double h, int bc, const double *d,
                        double dtau, int x, int y, int z)
{
    const size_t i = idx3(nx, ny, x, y, z);
    const double di = d[i];
    if (di == 0.0) return di;
    double dmx, dpx, dmy, dpy, dmz, dpz;
    one_sided(d, i, 1, x, nx, h, bc, &dmx, &dpx);
    one_sided(d, i, (size_t)nx, y, ny, h, bc, &dmy, &dpy);
    one_sided(d, i, (size_t)nx * (size_t)ny, z, nz, h, bc, &dmz, &dpz);
    double g;
    if (di > 0.0) {
        const double ax = max0(dmx), bx = min0(dpx);
        const double ay = max0(dmy), by = min0(dpy);
        const double az = max0(dmz), bz = min0(dpz);
        g = sqrt(((ax * ax + bx * bx) + (ay * ay + by * by)) + (az * az + bz * bz));
    } else {
        const double cx = max0(dpx), ex = min0(dmx);
        const double cy = max0(dpy), ey = min0(dmy);
        const double cz = max0(dpz), ez = min0(dmz);
        g = sqrt(((cx * cx + ex * ex) + (cy * cy + ey * ey)) + (cz * cz + ez * ez));
    }
    const double S = di / sqrt(di * di + (g * g) * (h * h));
    return di - dtau * (S * (g - 1.0));
}

/* One iteration of Eq. 12 on the points with nmask set (every point when
 * nmask is NULL); the others are copied. */
void orc_reinit_iter(int nx, int ny, int nz, double h, int bc, const double *d,
                     const uint8_t *nmask, double dtau, double *out)
{
    int z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t i = idx3(nx, ny, x, y, z);
                if (nmask && !nmask[i]) {
                    out[i] = d[i];
                    continue;
                }
                out[i] = orc_reinit_point(nx, ny, nz, h, bc, d, dtau, x, y, z);
            }
}

/* Eq. 10 on the points with nmask set (every point when nmask is NULL). */
void orc_clamp(int64_t n, double *d, const uint8_t *nmask, double gamma)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        if (nmask && !nmask[i]) continue;
        if (d[i] < -gamma) d[i] = -gamma;
        else if (d[i] > gamma) d[i] = gamma;
    }
}

/* One step of the local scheme: N from phi^n (Eq. 11), the cut-off advance
 * (Eq. 8) to phi-bar, `iters` iterations of Eq. 12 on N starting from
 * phi-bar, and the clamp of Eq. 10 on N.  work: 2 * n doubles, nmask_out:
 * n bytes (the N of this step). */
void orc_local_step(int nx, int ny, int nz, double h, int bc, const double *phi,
                    const double *F, double Fc, double beta, double gamma, double dt,
                    int iters, double dtau, double *out, double *work, uint8_t *nmask_out)
{
    const size_t n = (size_t)nx * ny * nz;
    double *a = work, *b = work + n;
    orc_region_n(nx, ny, nz, phi, gamma, nmask_out);
    orc_cut_step(nx, ny, nz, h, bc, phi, F, Fc, beta, gamma, dt, a);
    for (int m = 0; m < iters; ++m) {
        orc_reinit_iter(nx, ny, nz, h, bc, a, nmask_out, dtau, b);
        double *t = a;
        a = b;
        b = t;
    }
    orc_clamp((int64_t)n, a, nmask_out, gamma);
    memcpy(out, a, n * sizeof(double));
}
