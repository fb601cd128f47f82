/*
 * FP64 CPU oracle for motion-compensated SPDHG -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code, header, table or constant with the
 * CUDA path in paper_2410_10503_gb300/ and is written to be read against the
 * paper, not to be fast: one thread, plain loops, double precision.
 *
 * Operators of the gated data model d_i = A D_i x + eps_i (Sec. II-A):
 *   A      2D parallel-beam ray transform, Joseph's method, ray-driven.
 *   A^T    its adjoint, written as a ray-driven SCATTER over the same
 *          samples (independent of the GPU's pixel-driven gather).
 *   D_i    bilinear pull-back warp (rigid rotation+shift or dense field).
 *   D_i^T  scatter of the same bilinear taps (exact matrix transpose).
 * Gate draw of Algorithm 1 step (ii): Philox4x32-10 (Salmon et al., SC'11),
 * written from the published description.
 *
 * Geometry (the paper only says "2D parallel geometry", Sec. III):
 *   pixel (r, c) has centre (x, y) = (c - h, r - h), h = (n-1)/2, unit size;
 *   bin b has centre s_b = b - hb, hb = (nb-1)/2;  angle phi_k = k*pi/na;
 *   ray (k, b) = { p : p . (cos phi_k, sin phi_k) = s_b }.
 *   x-driven rays (n_a <= 4k <= 3 n_a, i.e. |sin| >= |cos|) are sampled once
 *   per image column with step 1/|sin|; the others once per row with step
 *   1/|cos|; linear interpolation between the two neighbouring pixels of
 *   that column (row), zero outside the image.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Angle k is sampled along columns ("x-driven") iff n_a <= 4k <= 3 n_a.
 * Integer rule so that 45 / 135 degrees are decided without rounding. */
static int x_driven(int k, int na) { return (na <= 4 * k) && (4 * k <= 3 * na); }

/* (A x)(k, b) = Delta_k * sum over driving lines of lerp(x) at the ray.
 * x: n*n row-major [r*n + c];  y: na*nb row-major [k*nb + b]. */
void or_ray_transform(int n, int na, int nb, const double* x, double* y)
{
    const double h = 0.5 * (n - 1), hb = 0.5 * (nb - 1);
    for (int k = 0; k < na; ++k) {
        const double phi = (double)k * M_PI / (double)na;
        const double cs = cos(phi), sn = sin(phi);
        for (int b = 0; b < nb; ++b) {
            const double s = (double)b - hb;
            double acc = 0.0, delta;
            if (x_driven(k, na)) {
                delta = 1.0 / fabs(sn);
                for (int c = 0; c < n; ++c) {
                    const double xc = (double)c - h;
                    const double rf = (s - xc * cs) / sn + h;   /* row coordinate */
                    const double r0 = floor(rf);
                    const double f = rf - r0;
                    const int i0 = (int)r0;
                    if (i0 >= 0 && i0 < n) acc += (1.0 - f) * x[(size_t)i0 * n + c];
                    if (i0 + 1 >= 0 && i0 + 1 < n) acc += f * x[(size_t)(i0 + 1) * n + c];
                }
            } else {
                delta = 1.0 / fabs(cs);
                for (int r = 0; r < n; ++r) {
                    const double yr = (double)r - h;
                    const double cf = (s - yr * sn) / cs + h;   /* column coordinate */
                    const double c0 = floor(cf);
                    const double f = cf - c0;
                    const int j0 = (int)c0;
                    if (j0 >= 0 && j0 < n) acc += (1.0 - f) * x[(size_t)r * n + j0];
                    if (j0 + 1 >= 0 && j0 + 1 < n) acc += f * x[(size_t)r * n + j0 + 1];
                }
            }
            y[(size_t)k * nb + b] = delta * acc;
        }
    }
}

/* A^T y by scattering every sample of every ray back onto its two pixels. */
void or_ray_transform_adj(int n, int na, int nb, const double* y, double* x)
{
    const double h = 0.5 * (n - 1), hb = 0.5 * (nb - 1);
    memset(x, 0, sizeof(double) * (size_t)n * n);
    for (int k = 0; k < na; ++k) {
        const double phi = (double)k * M_PI / (double)na;
        const double cs = cos(phi), sn = sin(phi);
        for (int b = 0; b < nb; ++b) {
            const double s = (double)b - hb;
            if (x_driven(k, na)) {
                const double v = y[(size_t)k * nb + b] / fabs(sn);
                for (int c = 0; c < n; ++c) {
                    const double xc = (double)c - h;
                    const double rf = (s - xc * cs) / sn + h;
                    const double r0 = floor(rf);
                    const double f = rf - r0;
                    const int i0 = (int)r0;
                    if (i0 >= 0 && i0 < n) x[(size_t)i0 * n + c] += (1.0 - f) * v;
                    if (i0 + 1 >= 0 && i0 + 1 < n) x[(size_t)(i0 + 1) * n + c] += f * v;
                }
            } else {
                const double v = y[(size_t)k * nb + b] / fabs(cs);
                for (int r = 0; r < n; ++r) {
                    const double yr = (double)r - h;
                    const double cf = (s - yr * sn) / cs + h;
                    const double c0 = floor(cf);
                    const double f = cf - c0;
                    const int j0 = (int)c0;
                    if (j0 >= 0 && j0 < n) x[(size_t)r * n + j0] += (1.0 - f) * v;
                    if (j0 + 1 >= 0 && j0 + 1 < n) x[(size_t)r * n + j0 + 1] += f * v;
                }
            }
        }
    }
}

/* Sample position of output pixel (r, c) under motion state i, in index
 * coordinates (row rq, column cq).  Rigid: q = R(phi) p + t about the image
 * centre, p = (c - h, r - h).  Dense: q = p + u(p) with u = (ux, uy) given
 * per pixel (field layout [2][n][n], channel 0 = ux). */
static void warp_point(int n, double phi, double tx, double ty, const float* field,
                       int r, int c, double* rq, double* cq)
{
    if (field) {
        const size_t p = (size_t)r * n + c;
        *cq = (double)c + (double)field[p];
        *rq = (double)r + (double)field[(size_t)n * n + p];
    } else {
        const double h = 0.5 * (n - 1);
        const double px = (double)c - h, py = (double)r - h;
        *cq = cos(phi) * px - sin(phi) * py + tx + h;
        *rq = sin(phi) * px + cos(phi) * py + ty + h;
    }
}

/* (D x)(p) = bilinear interpolation of x at q(p), zero outside the image.
 * field == NULL selects the rigid map (phi, tx, ty). */
void or_warp(int n, double phi, double tx, double ty, const float* field,
             const double* x, double* out)
{
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            double rq, cq;
            warp_point(n, phi, tx, ty, field, r, c, &rq, &cq);
            const double r0 = floor(rq), c0 = floor(cq);
            const double fr = rq - r0, fc = cq - c0;
            const int i0 = (int)r0, j0 = (int)c0;
            double acc = 0.0;
            for (int di = 0; di < 2; ++di)
                for (int dj = 0; dj < 2; ++dj) {
                    const int i = i0 + di, j = j0 + dj;
                    const double w = (di ? fr : 1.0 - fr) * (dj ? fc : 1.0 - fc);
                    if (i >= 0 && i < n && j >= 0 && j < n) acc += w * x[(size_t)i * n + j];
                }
            out[(size_t)r * n + c] = acc;
        }
}

/* D^T v: every output pixel p of D scatters v(p) onto its four taps. */
void or_warp_adj(int n, double phi, double tx, double ty, const float* field,
                 const double* v, double* out)
{
    memset(out, 0, sizeof(double) * (size_t)n * n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            double rq, cq;
            warp_point(n, phi, tx, ty, field, r, c, &rq, &cq);
            const double r0 = floor(rq), c0 = floor(cq);
            const double fr = rq - r0, fc = cq - c0;
            const int i0 = (int)r0, j0 = (int)c0;
            const double val = v[(size_t)r * n + c];
            for (int di = 0; di < 2; ++di)
                for (int dj = 0; dj < 2; ++dj) {
                    const int i = i0 + di, j = j0 + dj;
                    const double w = (di ? fr : 1.0 - fr) * (dj ? fc : 1.0 - fc);
                    if (i >= 0 && i < n && j >= 0 && j < n) out[(size_t)i * n + j] += w * val;
                }
        }
}

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------
 * Round: two 32x32->64 products of counter words 0 and 2 with the published
 * multipliers; the new counter is (hi1^c1^k0, lo1, hi0^c3^k1, lo0).  The key
 * is bumped by the two Weyl constants between rounds. */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k[0];
    const uint32_t n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k[1];
    const uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* First output word for iteration k: key = seed, counter = (k_lo, stream, k_hi, 0). */
static uint32_t gate_word(uint64_t seed, uint32_t stream, uint64_t k)
{
    const uint32_t ctr[4] = {(uint32_t)k, stream, (uint32_t)(k >> 32), 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[0];
}

/* Serial sampling, one gate per iteration (Algorithm 1 step (ii)).
 * thresholds == NULL: uniform p_i = 1/N, gate = floor(word * N / 2^32).
 * Otherwise thresholds[i] = floor(2^32 * (p_0 + ... + p_i)) (last = 2^32) and
 * the gate is the first i with word < thresholds[i]. */
void or_draw_gates(uint64_t seed, uint32_t stream, uint64_t k0, int count, int n_gates,
                   const uint64_t* thresholds, int32_t* out)
{
    for (int j = 0; j < count; ++j) {
        const uint32_t w = gate_word(seed, stream, k0 + (uint64_t)j);
        if (!thresholds) {
            out[j] = (int32_t)(((uint64_t)w * (uint64_t)n_gates) >> 32);
        } else {
            int g = 0;
            while (g < n_gates - 1 && (uint64_t)w >= thresholds[g]) ++g;
            out[j] = g;
        }
    }
}

/* Vector-Jacobian product of the dense-field warp: for (D_u x)(p) =
 * bilinear(x)(p + u(p)), out[0][p] = g(p) d(D_u x)(p)/du_x(p) and
 * out[1][p] = g(p) d(D_u x)(p)/du_y(p).  The derivative is that of the
 * bilinear interpolant inside the cell holding q(p) (taps outside the image
 * are zero), i.e. one-sided on the cell's lower edges. */
void or_warp_field_vjp(int n, const float* field, const double* x, const double* g, double* out)
{
    const size_t n2 = (size_t)n * n;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            const size_t p = (size_t)r * n + c;
            const double cq = (double)c + (double)field[p];
            const double rq = (double)r + (double)field[n2 + p];
            const double r0 = floor(rq), c0 = floor(cq);
            const double fr = rq - r0, fc = cq - c0;
            const int i0 = (int)r0, j0 = (int)c0;
            double v[2][2];
            for (int di = 0; di < 2; ++di)
                for (int dj = 0; dj < 2; ++dj) {
                    const int i = i0 + di, j = j0 + dj;
                    v[di][dj] = (i >= 0 && i < n && j >= 0 && j < n) ? x[(size_t)i * n + j] : 0.0;
                }
            const double dcol = (1.0 - fr) * (v[0][1] - v[0][0]) + fr * (v[1][1] - v[1][0]);
            const double drow = (1.0 - fc) * (v[1][0] - v[0][0]) + fc * (v[1][1] - v[0][1]);
            out[p] = g[p] * dcol;
            out[n2 + p] = g[p] * drow;
        }
}
