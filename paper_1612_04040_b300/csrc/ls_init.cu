// ls_init.cu -- Step 0 of the narrow-band algorithm (section 1.1): the
// initial level-set function phi(x, 0) = +-d (Eq. 1) and speed fields,
// evaluated in FP64 on the device at the cell centres ((i+1/2) h, ...) and
// stored in the context's precision directly in the bricked layout.
//
// Shapes (phi < 0 inside):
//   LS_SHAPE_SPHERES  params = [n, (cx, cy, cz, r) x n]: min_i |x - c_i| - r_i
//   LS_SHAPE_TORUS    params = [cx, cy, cz, ax, ay, az, R, r] (unit axis a):
//                     sqrt((rho - R)^2 + s^2) - r, s = (x-c).a, rho = |x-c - s a|
//   LS_SHAPE_SH       params = [cx, cy, cz, base, amp, lmax, a_lm...]:
//                     |x - c| - (base + amp * sum_lm a_lm Y_lm(direction)),
//                     Y_lm the real orthonormal spherical harmonics
//                     N_lm P_l^|m|(cos t) T_m(p), T_m = sqrt2 cos(m p) (m > 0),
//                     1 (m = 0), sqrt2 sin(|m| p) (m < 0), with
//                     N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) computed
//                     here; modes ordered l = 1..lmax, m = -l..l
// Speeds:
//   LS_SPEED_SINUSOID 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z)
//   LS_SPEED_COSCOS   cos(4 pi x) cos(4 pi y)
//   LS_SPEED_FOURIER  params = [n, (a, kx, ky, kz, theta) x n]:
//                     sum a cos(2 pi k.x + theta) / sum |a|
#include <math.h>

#include "ls.h"
#include "ls_internal.cuh"

namespace lsk {

namespace {

constexpr double PI = 3.14159265358979323846;

__device__ double sh_radius(const double* p, double ux, double uy, double uz)
{
    const double base = p[3], amp = p[4];
    const int lmax = (int)p[5];
    const double* a = p + 6;
    const double ct = fmin(fmax(uz, -1.0), 1.0);
    const double st = sqrt(fmax(1.0 - ct * ct, 0.0));
    const double ph = atan2(uy, ux);
    double s = 0.0;
    // P_l^m by the standard recurrences (no Condon-Shortley phase); the
    // normalisation N_lm from the factorial ratio (l+m)!/(l-m)!, carried
    // along l for fixed m: ratio(m, m) = (2m)!, ratio(l+1, m) = ratio(l, m)
    // (l+1+m)/(l+1-m)
    for (int m = 0; m <= lmax; ++m) {
        double pmm = 1.0, fact = 1.0, ratio = 1.0;
        for (int k = 0; k < m; ++k) {
            pmm = pmm * fact * st;
            fact += 2.0;
        }
        for (int k = 2; k <= 2 * m; ++k) ratio *= (double)k;
        const double tm = m > 0 ? sqrt(2.0) : 1.0;
        double p_lm2 = 0.0, p_lm1 = 0.0;
        for (int l = m; l <= lmax; ++l) {
            double plm;
            if (l == m) plm = pmm;
            else if (l == m + 1) plm = ct * (2 * m + 1) * pmm;
            else plm = ((2 * l - 1) * ct * p_lm1 - (l + m - 1) * p_lm2) / (l - m);
            p_lm2 = p_lm1;
            p_lm1 = plm;
            if (l > m) ratio *= (double)(l + m) / (double)(l - m);
            if (l < 1) continue;
            const double nrm = tm * sqrt((2 * l + 1) / (4.0 * PI) / ratio);
            const int base_idx = l * l - 1;  // index of (l, m = -l)
            if (m == 0) {
                s += a[base_idx + l] * nrm * plm;
            } else {
                s += a[base_idx + l + m] * nrm * plm * cos(m * ph);
                s += a[base_idx + l - m] * nrm * plm * sin(m * ph);
            }
        }
    }
    return base + amp * s;
}

__device__ double shape_value(int kind, const double* p, double x, double y, double z)
{
    if (kind == LS_SHAPE_SPHERES) {
        const int n = (int)p[0];
        double best = 1e300;
        for (int i = 0; i < n; ++i) {
            const double* q = p + 1 + 4 * i;
            const double dx = x - q[0], dy = y - q[1], dz = z - q[2];
            const double d = sqrt(dx * dx + dy * dy + dz * dz) - q[3];
            best = d < best ? d : best;
        }
        return best;
    }
    if (kind == LS_SHAPE_TORUS) {
        const double px = x - p[0], py = y - p[1], pz = z - p[2];
        const double s = px * p[3] + py * p[4] + pz * p[5];
        const double qx = px - s * p[3], qy = py - s * p[4], qz = pz - s * p[5];
        const double rho = sqrt(qx * qx + qy * qy + qz * qz);
        return sqrt((rho - p[6]) * (rho - p[6]) + s * s) - p[7];
    }
    // LS_SHAPE_SH
    const double px = x - p[0], py = y - p[1], pz = z - p[2];
    const double rr = sqrt(px * px + py * py + pz * pz);
    return rr - sh_radius(p, px / rr, py / rr, pz / rr);
}

__device__ double speed_value(int kind, const double* p, double x, double y, double z)
{
    if (kind == LS_SPEED_SINUSOID)
        return 1.0 + 0.5 * sin(2.0 * PI * x) * sin(2.0 * PI * y) * sin(2.0 * PI * z);
    if (kind == LS_SPEED_COSCOS) return cos(4.0 * PI * x) * cos(4.0 * PI * y);
    // LS_SPEED_FOURIER
    const int n = (int)p[0];
    double s = 0.0, norm = 0.0;
    for (int i = 0; i < n; ++i) {
        const double* q = p + 1 + 5 * i;
        s += q[0] * cos(2.0 * PI * (q[1] * x + q[2] * y + q[3] * z) + q[4]);
        norm += fabs(q[0]);
    }
    return s / (norm > 0.0 ? norm : 1.0);
}

// one thread per grid point of one instance, written in bricked order
template <typename T>
__global__ void k_init_field(T* __restrict__ out, T* __restrict__ out2, Inst in, int is_speed,
                             int kind, const double* __restrict__ p)
{
    const long long n = in.ntiles * TILE_PTS;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long t = e / TILE_PTS;
        const int r = (int)(e - t * TILE_PTS);
        const int lx = r & 7, ly = (r >> 3) & 7, lz = r >> 6;
        const long long tpl = (long long)in.tnx * in.tny;
        const int tz = (int)(t / tpl);
        const int rem = (int)(t - (long long)tz * tpl);
        const int ty = rem / in.tnx, tx = rem - ty * in.tnx;
        const double x = (tx * 8 + lx + 0.5) * in.h;
        const double y = (ty * 8 + ly + 0.5) * in.h;
        const double z = (tz * 8 + lz + 0.5) * in.h;
        const double v = is_speed ? speed_value(kind, p, x, y, z) : shape_value(kind, p, x, y, z);
        out[e] = (T)v;
        if (out2) out2[e] = (T)v;
    }
}

}  // namespace

cudaError_t launch_init_field(void* out, void* out2, const Inst& in, int prec, int is_speed,
                              int kind, const double* params, cudaStream_t s)
{
    const long long n = in.ntiles * TILE_PTS;
    long long g = (n + 255) / 256;
    if (g > 148 * 32) g = 148 * 32;
    if (prec == 0)
        k_init_field<float><<<(int)g, 256, 0, s>>>((float*)out, (float*)out2, in, is_speed, kind, params);
    else
        k_init_field<double><<<(int)g, 256, 0, s>>>((double*)out, (double*)out2, in, is_speed, kind,
                                                     params);
    return cudaGetLastError();
}

}  // namespace lsk
