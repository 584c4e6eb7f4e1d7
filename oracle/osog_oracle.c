/*
 * FP64 CPU oracle for the OSOG optical forward model (arxiv 2606.21381).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls
 * this file; only the tests, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA path: every quantity here is computed from its plain definition
 * in double precision, slowly and in the paper's order.
 *
 * What it computes (paper sections / equations):
 *   - particle geometry: ellipsoids (quadric chord), bevelled rectangular
 *     prisms as an intersection of M = 14 half-spaces, P = {x : A x <= b}
 *     (Sec. III.A, Eq. 1), and general convex polyhedra given by the
 *     caller's own M planes (kind 2, Eq. 1);
 *   - OPD and absorption maps: sum over particles of dn_p * t_p and
 *     mu_p * t_p, overlaps add (Eq. 2's integral over z; Eq. 7's
 *     accumulate=True composition, Sec. III.C);
 *   - exit wave E = exp(-ATT) * exp(i 2 pi OPD / lambda) (Eq. 2, Beer-Lambert
 *     amplitude of Eq. 4);
 *   - pupil P(k) = circ(|k|/k_NA) exp(i dz (sqrt(k0^2 - |k|^2) - k0)) (Eq. 3)
 *     and the coherent image I = |E * h_obj|^2 (Sec. III.B, brightfield);
 *     oblique illumination as the pupil shifted by k_ill (Fig. 2 discussion:
 *     "asymmetric Fourier pupil"); DIC as the sheared-field difference of
 *     Eq. 5 taken coherently through the pupil, and in the literal
 *     incoherent reading of Eq. 5 (orc_dic_incoherent);
 *   - an own radix-2 FFT and a brute-force DFT (used to pin the FFT);
 *   - the losses of inverse rendering: the log-amplitude spectral loss of
 *     Eq. 8 (orc_spectral_loss) and the low-pass image misfit of the
 *     coarse-to-fine solve (orc_lowpass_misfit), each with its gradient
 *     with respect to the image;
 *   - the gradient of a linear functional of the images with respect to
 *     every particle field and to the optics scalars, by the analytic
 *     adjoint of the chain above (orc_render_grad), pinned by central
 *     finite differences of orc_render.
 *
 * Conventions (readings of points the paper leaves open):
 *   - pixel (i, j) is sampled at its centre (x, y) = (j + 0.5, i + 0.5) px;
 *   - local frame u = c (x - cx) + s (y - cy), v = -s (x - cx) + c (y - cy);
 *   - ellipsoid: in-plane semi-axes a, b (px), full central thickness T (um);
 *   - prism: half-lengths hx, hy (px), thickness T (um), chamfer planes of
 *     slope s_b on all top and bottom edges meeting at zero wall height;
 *   - forward DFT kernel exp(-2 pi i jk/N); inverse unnormalised, the
 *     image carries 1/(H W);
 *   - k grid 2 pi * fftfreq(N, dx); k0 = 2 pi n_m / lambda.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Field order of the structure-of-arrays particle tensor, row by row. */
enum { F_CX = 0, F_CY, F_TH, F_A, F_B, F_T, F_DN, F_MU, F_KIND, F_COUNT };

typedef struct {
    int32_t H, W;
    double dx;            /* pixel pitch, um */
    double lambda;        /* wavelength, um */
    double NA;
    double n_medium;
    double defocus;       /* dz, um */
    uint32_t modes;       /* bit 0 brightfield, bit 1 oblique, bit 2 DIC */
    double oblique_frac;  /* |k_ill| = frac * k_NA */
    double oblique_angle; /* direction of k_ill, rad */
    double shear_px;      /* 2 |ds| in px */
    double shear_angle;   /* direction of ds, rad */
    double bias_phase;    /* theta of Eq. 5 */
    double bevel_slope;   /* s_b of the prism chamfers */
} orc_optics;

/* ------------------------------------------------------------------ */
/* Geometry                                                            */
/* ------------------------------------------------------------------ */

/* Chord length (um) of the vertical line through local point (u, v) (um)
 * inside the convex polyhedron {x : A x <= b}: the z-interval bounded by
 * every half-space, Eq. 1.  A is m x 3 row-major. */
double orc_halfspace_chord(const double *A, const double *b, int m,
                           double u, double v)
{
    double zlo = -INFINITY, zhi = INFINITY;
    for (int i = 0; i < m; ++i) {
        double ax = A[3 * i], ay = A[3 * i + 1], az = A[3 * i + 2];
        double rhs = b[i] - ax * u - ay * v;
        if (az > 0.0) {
            double z = rhs / az;
            if (z < zhi) zhi = z;
        } else if (az < 0.0) {
            double z = rhs / az;
            if (z > zlo) zlo = z;
        } else if (rhs < 0.0) {
            return 0.0;
        }
    }
    return zhi > zlo ? zhi - zlo : 0.0;
}

/* The 14 half-spaces of a bevelled rectangular prism in its local frame
 * (um): top and bottom faces, four side walls, and eight chamfers of slope
 * s on the top and bottom edges.  Writes A (14 x 3) and b (14). */
void orc_prism_halfspaces(double hx_um, double hy_um, double T, double s,
                          double *A, double *b)
{
    const double h = 0.5 * T;
    double rows[14][4] = {
        { 0, 0, 1, h},  { 0, 0, -1, h},
        { 1, 0, 0, hx_um}, {-1, 0, 0, hx_um},
        { 0, 1, 0, hy_um}, { 0, -1, 0, hy_um},
        { s, 0, 1, s * hx_um}, {-s, 0, 1, s * hx_um},
        { 0, s, 1, s * hy_um}, { 0, -s, 1, s * hy_um},
        { s, 0, -1, s * hx_um}, {-s, 0, -1, s * hx_um},
        { 0, s, -1, s * hy_um}, { 0, -s, -1, s * hy_um},
    };
    for (int i = 0; i < 14; ++i) {
        A[3 * i] = rows[i][0];
        A[3 * i + 1] = rows[i][1];
        A[3 * i + 2] = rows[i][2];
        b[i] = rows[i][3];
    }
}

/* Planes of the general polyhedra (kind 2): particle p owns rows
 * off[p] .. off[p+1]-1 of planes, each (a_x, a_y, a_z, b) of one half-space
 * a . (u, v, z) <= b in the particle's local frame (um). */
typedef struct {
    const double *planes;
    const int32_t *off;
} orc_planes;

/* Thickness t (um) of particle p (fields widened from fp32) at the canvas
 * point (x, y) px. */
static double particle_thickness(const double *q, int p, const orc_planes *pl,
                                 double dx, double bevel, double x, double y)
{
    double c = cos(q[F_TH]), s = sin(q[F_TH]);
    double ex = x - q[F_CX], ey = y - q[F_CY];
    double u = c * ex + s * ey;
    double v = -s * ex + c * ey;
    if (q[F_KIND] > 1.5) {
        if (!pl || !pl->planes) return 0.0;
        int m = pl->off[p + 1] - pl->off[p];
        double A[3 * 64], b[64];
        if (m > 64) m = 64;
        for (int i = 0; i < m; ++i) {
            const double *r = pl->planes + 4 * (size_t)(pl->off[p] + i);
            A[3 * i] = r[0];
            A[3 * i + 1] = r[1];
            A[3 * i + 2] = r[2];
            b[i] = r[3];
        }
        return orc_halfspace_chord(A, b, m, u * dx, v * dx);
    }
    if (q[F_KIND] > 0.5) {
        double A[42], b[14];
        orc_prism_halfspaces(q[F_A] * dx, q[F_B] * dx, q[F_T], bevel, A, b);
        return orc_halfspace_chord(A, b, 14, u * dx, v * dx);
    }
    double ua = u / q[F_A], vb = v / q[F_B];
    double r = 1.0 - ua * ua - vb * vb;
    return r > 0.0 ? q[F_T] * sqrt(r) : 0.0;
}

static void load_particle(const float *soa, int64_t ld, int p, double *q)
{
    for (int f = 0; f < F_COUNT; ++f) q[f] = (double)soa[(int64_t)f * ld + p];
}

/* OPD and absorption-thickness maps (H x W, row-major), Eq. 2 / Eq. 7:
 * opd(x, y) = sum_p dn_p t_p(x, y), att(x, y) = sum_p mu_p t_p(x, y), with
 * particles added in ascending index.  Each particle is evaluated on the
 * pixels of its circumscribed square plus one pixel (t is zero outside it)
 * unless full_canvas is set, in which case every pixel is evaluated. */
static void opd_att_planes(const float *soa, int64_t ld, int n, int H, int W,
                           double dx, double bevel, int full_canvas,
                           const orc_planes *pl, double *opd, double *att)
{
    memset(opd, 0, sizeof(double) * (size_t)H * W);
    memset(att, 0, sizeof(double) * (size_t)H * W);
    for (int p = 0; p < n; ++p) {
        double q[F_COUNT];
        load_particle(soa, ld, p, q);
        int j0 = 0, j1 = W - 1, i0 = 0, i1 = H - 1;
        if (!full_canvas) {
            /* kind 2: a is the footprint's circumscribed radius (px) */
            double R = q[F_KIND] > 1.5 ? q[F_A]
                     : q[F_KIND] > 0.5 ? sqrt(q[F_A] * q[F_A] + q[F_B] * q[F_B])
                                       : fmax(q[F_A], q[F_B]);
            double jl = floor(q[F_CX] - R - 1.5), jh = ceil(q[F_CX] + R + 0.5);
            double il = floor(q[F_CY] - R - 1.5), ih = ceil(q[F_CY] + R + 0.5);
            if (jh < 0 || ih < 0 || jl > W - 1 || il > H - 1) continue;
            j0 = jl < 0 ? 0 : (int)jl;
            j1 = jh > W - 1 ? W - 1 : (int)jh;
            i0 = il < 0 ? 0 : (int)il;
            i1 = ih > H - 1 ? H - 1 : (int)ih;
        }
        for (int i = i0; i <= i1; ++i)
            for (int j = j0; j <= j1; ++j) {
                double t = particle_thickness(q, p, pl, dx, bevel, j + 0.5, i + 0.5);
                if (t != 0.0) {
                    opd[(size_t)i * W + j] += q[F_DN] * t;
                    att[(size_t)i * W + j] += q[F_MU] * t;
                }
            }
    }
}

void orc_opd_att(const float *soa, int64_t ld, int n, int H, int W,
                 double dx, double bevel, int full_canvas,
                 double *opd, double *att)
{
    opd_att_planes(soa, ld, n, H, W, dx, bevel, full_canvas, NULL, opd, att);
}

/* As orc_opd_att with the plane sets of kind-2 particles (planes: rows of
 * (a_x, a_y, a_z, b); off: [n + 1] row offsets). */
void orc_opd_att_poly(const float *soa, int64_t ld, int n, int H, int W,
                      double dx, double bevel, int full_canvas,
                      const double *planes, const int32_t *off,
                      double *opd, double *att)
{
    orc_planes pl = {planes, off};
    opd_att_planes(soa, ld, n, H, W, dx, bevel, full_canvas, &pl, opd, att);
}

/* OPD at a list of pixels by brute force over every particle (no window):
 * an independent route to single samples of a large canvas. */
void orc_opd_at(const float *soa, int64_t ld, int n, double dx, double bevel,
                const int64_t *pix, int64_t npix, int W, double *opd,
                double *att)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < npix; ++k) {
        int i = (int)(pix[k] / W), j = (int)(pix[k] % W);
        double so = 0.0, sa = 0.0;
        for (int p = 0; p < n; ++p) {
            double q[F_COUNT];
            load_particle(soa, ld, p, q);
            double t = particle_thickness(q, p, NULL, dx, bevel, j + 0.5, i + 0.5);
            so += q[F_DN] * t;
            sa += q[F_MU] * t;
        }
        opd[k] = so;
        att[k] = sa;
    }
}

/* Exit wave, Eq. 2 with the Beer-Lambert amplitude of Eq. 4:
 * E = exp(-att) * (cos, sin)(2 pi opd / lambda). */
void orc_field(const double *opd, const double *att, int64_t count,
               double lambda, double *re, double *im)
{
    for (int64_t k = 0; k < count; ++k) {
        double a = exp(-att[k]);
        double ph = 2.0 * M_PI * opd[k] / lambda;
        re[k] = a * cos(ph);
        im[k] = a * sin(ph);
    }
}

/* ------------------------------------------------------------------ */
/* Fourier transforms                                                  */
/* ------------------------------------------------------------------ */

/* In-place radix-2 decimation-in-time FFT of one line of n points (n a
 * power of two) with stride 1: bit-reversal permutation, then log2(n)
 * butterfly stages with twiddles exp(sign 2 pi i k / len).  Unnormalised. */
static void fft_line(double *re, double *im, int n, int sign)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; ++k) {
            double ang = sign * 2.0 * M_PI * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + k, b = s + k + half;
                double tr = re[b] * wr - im[b] * wi;
                double ti = re[b] * wi + im[b] * wr;
                re[b] = re[a] - tr; im[b] = im[a] - ti;
                re[a] += tr;        im[a] += ti;
            }
        }
    }
}

/* 2-D FFT of an H x W row-major array: every row, then every column.
 * sign = -1 forward, +1 inverse; unnormalised. */
void orc_fft2(double *re, double *im, int H, int W, int sign)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i) fft_line(re + (size_t)i * W, im + (size_t)i * W, W, sign);
#pragma omp parallel
    {
        double *cr = (double *)malloc(sizeof(double) * H);
        double *ci = (double *)malloc(sizeof(double) * H);
#pragma omp for schedule(static)
        for (int j = 0; j < W; ++j) {
            for (int i = 0; i < H; ++i) { cr[i] = re[(size_t)i * W + j]; ci[i] = im[(size_t)i * W + j]; }
            fft_line(cr, ci, H, sign);
            for (int i = 0; i < H; ++i) { re[(size_t)i * W + j] = cr[i]; im[(size_t)i * W + j] = ci[i]; }
        }
        free(cr);
        free(ci);
    }
}

/* Brute-force 2-D DFT straight from its definition, O((HW)^2):
 * X[k, l] = sum_{i, j} x[i, j] exp(sign 2 pi i (k i / H + l j / W)). */
void orc_dft2_brute(const double *re, const double *im, int H, int W, int sign,
                    double *ore, double *oim)
{
    for (int k = 0; k < H; ++k)
        for (int l = 0; l < W; ++l) {
            double sr = 0.0, si = 0.0;
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    double ang = sign * 2.0 * M_PI *
                                 ((double)((int64_t)k * i % H) / H + (double)((int64_t)l * j % W) / W);
                    double c = cos(ang), s = sin(ang);
                    double xr = re[(size_t)i * W + j], xi = im[(size_t)i * W + j];
                    sr += xr * c - xi * s;
                    si += xr * s + xi * c;
                }
            ore[(size_t)k * W + l] = sr;
            oim[(size_t)k * W + l] = si;
        }
}

/* ------------------------------------------------------------------ */
/* Optical head                                                        */
/* ------------------------------------------------------------------ */

/* Angular spatial frequency of DFT index idx on an n-point grid of pitch
 * dx: 2 pi * fftfreq(n, dx)[idx]. */
static double kfreq(int idx, int n, double dx)
{
    int f = idx < n / 2 ? idx : idx - n;
    return 2.0 * M_PI * (double)f / ((double)n * dx);
}

/* Pupil of Eq. 3 at angular frequency q: circ(|q| / k_NA) times the
 * defocus phase exp(i dz (sqrt(k0^2 - |q|^2) - k0)); the constant -k0 only
 * removes a global phase.  The circle is closed (|q| = k_NA is inside). */
static void pupil(const orc_optics *o, double qx, double qy, double *pr, double *pi)
{
    double kna = 2.0 * M_PI * o->NA / o->lambda;
    double k0 = 2.0 * M_PI * o->n_medium / o->lambda;
    double q2 = qx * qx + qy * qy;
    if (q2 > kna * kna) { *pr = 0.0; *pi = 0.0; return; }
    double chi = o->defocus * (sqrt(k0 * k0 - q2) - k0);
    *pr = cos(chi);
    *pi = sin(chi);
}

/* Transfer function H_m(k) on the H x W DFT grid for one modality:
 *   mode 1 brightfield:  P(k)
 *   mode 2 oblique:      P(k + k_ill), k_ill = frac k_NA (cos phi, sin phi)
 *   mode 4 DIC:          P(k) * 2i sin(k . ds + theta), ds = shear_px dx / 2
 *                        along shear_angle (Fourier transform of
 *                        U(r + ds) e^{i theta} - U(r - ds) e^{-i theta}). */
void orc_transfer(const orc_optics *o, int mode, double *hre, double *him)
{
    int H = o->H, W = o->W;
    double kna = 2.0 * M_PI * o->NA / o->lambda;
    double offx = 0.0, offy = 0.0;
    if (mode == 2) {
        offx = o->oblique_frac * kna * cos(o->oblique_angle);
        offy = o->oblique_frac * kna * sin(o->oblique_angle);
    }
    double dsx = 0.5 * o->shear_px * o->dx * cos(o->shear_angle);
    double dsy = 0.5 * o->shear_px * o->dx * sin(o->shear_angle);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double kx = kfreq(j, W, o->dx), ky = kfreq(i, H, o->dx);
            double pr, pi;
            pupil(o, kx + offx, ky + offy, &pr, &pi);
            if (mode == 4) {
                double g = 2.0 * sin(kx * dsx + ky * dsy + o->bias_phase);
                /* (pr + i pi) * (i g) */
                double r = -pi * g, m = pr * g;
                pr = r;
                pi = m;
            }
            hre[(size_t)i * W + j] = pr;
            him[(size_t)i * W + j] = pi;
        }
}

/* Images for every modality in o->modes (bit order: brightfield, oblique,
 * DIC) from an exit wave:  I_m = | IDFT2( DFT2(E) * H_m ) / (H W) |^2.
 * images is K x H x W.  The field arrays are left unchanged. */
void orc_images(const orc_optics *o, const double *ere, const double *eim,
                double *images)
{
    int H = o->H, W = o->W;
    size_t hw = (size_t)H * W;
    double *fr = (double *)malloc(sizeof(double) * hw);
    double *fi = (double *)malloc(sizeof(double) * hw);
    double *hr = (double *)malloc(sizeof(double) * hw);
    double *hi = (double *)malloc(sizeof(double) * hw);
    double *zr = (double *)malloc(sizeof(double) * hw);
    double *zi = (double *)malloc(sizeof(double) * hw);
    memcpy(fr, ere, sizeof(double) * hw);
    memcpy(fi, eim, sizeof(double) * hw);
    orc_fft2(fr, fi, H, W, -1);
    int k = 0;
    for (int bit = 0; bit < 3; ++bit) {
        int mode = 1 << bit;
        if (!(o->modes & (uint32_t)mode)) continue;
        orc_transfer(o, mode, hr, hi);
        for (size_t t = 0; t < hw; ++t) {
            zr[t] = fr[t] * hr[t] - fi[t] * hi[t];
            zi[t] = fr[t] * hi[t] + fi[t] * hr[t];
        }
        orc_fft2(zr, zi, H, W, +1);
        double inv = 1.0 / (double)hw;
        double *img = images + (size_t)k * hw;
        for (size_t t = 0; t < hw; ++t) {
            double a = zr[t] * inv, b = zi[t] * inv;
            img[t] = a * a + b * b;
        }
        ++k;
    }
    free(fr); free(fi); free(hr); free(hi); free(zr); free(zi);
}

/* DIC read literally from Eq. 5 (incoherent reading): the exit wave itself,
 * not the filtered field, is sheared and interfered,
 *   J(r) = | U(r + ds) e^{i theta} - U(r - ds) e^{-i theta} |^2,
 * computed as D = IDFT2( DFT2(U) * 2i sin(k . ds + theta) ) / (H W) (shift
 * theorem; every frequency, no pupil), and the intensity is then blurred by
 * the objective's intensity point spread function |h|^2, h = IDFT2(P) /
 * (H W) with P the brightfield pupil of Eq. 3 (NA, defocus), normalised to
 * unit sum so that a uniform J stays uniform:
 *   I = J (*) |h|^2 / sum |h|^2   (circular convolution, via the DFT).
 * out is H x W. */
void orc_dic_incoherent(const orc_optics *o, const double *ere, const double *eim,
                        double *out)
{
    int H = o->H, W = o->W;
    size_t N = (size_t)H * W;
    double *dr = (double *)malloc(sizeof(double) * N), *di = (double *)malloc(sizeof(double) * N);
    double *hr = (double *)malloc(sizeof(double) * N), *hi = (double *)malloc(sizeof(double) * N);
    double *jr = (double *)malloc(sizeof(double) * N), *ji = (double *)malloc(sizeof(double) * N);
    double dsx = 0.5 * o->shear_px * o->dx * cos(o->shear_angle);
    double dsy = 0.5 * o->shear_px * o->dx * sin(o->shear_angle);
    /* D and J = |D|^2 */
    memcpy(dr, ere, sizeof(double) * N);
    memcpy(di, eim, sizeof(double) * N);
    orc_fft2(dr, di, H, W, -1);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            size_t q = (size_t)i * W + j;
            double g = 2.0 * sin(kfreq(j, W, o->dx) * dsx + kfreq(i, H, o->dx) * dsy + o->bias_phase);
            double r = -di[q] * g, m = dr[q] * g; /* (dr + i di) * (i g) */
            dr[q] = r;
            di[q] = m;
        }
    orc_fft2(dr, di, H, W, +1);
    for (size_t q = 0; q < N; ++q) {
        double a = dr[q] / (double)N, b = di[q] / (double)N;
        jr[q] = a * a + b * b;
        ji[q] = 0.0;
    }
    /* |h|^2 of the brightfield pupil, normalised to unit sum */
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j)
            pupil(o, kfreq(j, W, o->dx), kfreq(i, H, o->dx), &hr[(size_t)i * W + j],
                  &hi[(size_t)i * W + j]);
    orc_fft2(hr, hi, H, W, +1);
    double sum = 0.0;
    for (size_t q = 0; q < N; ++q) {
        double a = hr[q] / (double)N, b = hi[q] / (double)N;
        hr[q] = a * a + b * b;
        hi[q] = 0.0;
        sum += hr[q];
    }
    for (size_t q = 0; q < N; ++q) hr[q] /= sum;
    /* circular convolution J (*) psf by the DFT */
    orc_fft2(jr, ji, H, W, -1);
    orc_fft2(hr, hi, H, W, -1);
    for (size_t q = 0; q < N; ++q) {
        double r = jr[q] * hr[q] - ji[q] * hi[q], m = jr[q] * hi[q] + ji[q] * hr[q];
        jr[q] = r;
        ji[q] = m;
    }
    orc_fft2(jr, ji, H, W, +1);
    for (size_t q = 0; q < N; ++q) out[q] = jr[q] / (double)N;
    free(dr); free(di); free(hr); free(hi); free(jr); free(ji);
}

/* Whole forward model f(Theta) = I: OPD/ATT maps, exit wave, images. */
void orc_render(const float *soa, int64_t ld, int n, const orc_optics *o,
                double *opd, double *att, double *ere, double *eim,
                double *images)
{
    orc_opd_att(soa, ld, n, o->H, o->W, o->dx, o->bevel_slope, 0, opd, att);
    orc_field(opd, att, (int64_t)o->H * o->W, o->lambda, ere, eim);
    orc_images(o, ere, eim, images);
}

/* orc_render with kind-2 particles and their planes. */
void orc_render_poly(const float *soa, int64_t ld, int n, const double *planes,
                     const int32_t *off, const orc_optics *o, double *opd,
                     double *att, double *ere, double *eim, double *images)
{
    orc_opd_att_poly(soa, ld, n, o->H, o->W, o->dx, o->bevel_slope, 0, planes,
                     off, opd, att);
    orc_field(opd, att, (int64_t)o->H * o->W, o->lambda, ere, eim);
    orc_images(o, ere, eim, images);
}

/* ------------------------------------------------------------------ */
/* Gradient (analytic adjoint, FP64)                                   */
/* ------------------------------------------------------------------ */

/* Chord of the bevelled prism at local point (u, v) (um) and its partial
 * derivatives, from the active half-spaces of Eq. 1: chord = z_top - z_bot
 * with z_top the lowest upper bound (planes with a_z > 0) and z_bot the
 * highest lower bound (a_z < 0), each z = (b - a_x u - a_y v) / a_z.  The
 * derivative follows the two active planes; b depends on (hx, hy, T) with
 * the partials of the 14 planes (top/bottom b = T/2, walls b = hx or hy,
 * chamfers b = s hx or s hy).  d[0..4] = d chord / d(u, v, hx, hy, T), all
 * in um.  Returns the chord (0 and zero partials outside). */
static double prism_chord_grad(double hx, double hy, double T, double s,
                               double u, double v, double d[5])
{
    double A[42], b[14];
    /* db/d(hx, hy, T) of each plane, in the order of orc_prism_halfspaces:
     * top, bottom (b = T/2); walls +-x (b = hx), +-y (b = hy); chamfers
     * top +-x, top +-y, bottom +-x, bottom +-y (b = s hx or s hy). */
    const double db[14][3] = {
        {0, 0, 0.5}, {0, 0, 0.5}, {1, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 1, 0},
        {s, 0, 0}, {s, 0, 0}, {0, s, 0}, {0, s, 0},
        {s, 0, 0}, {s, 0, 0}, {0, s, 0}, {0, s, 0}};
    orc_prism_halfspaces(hx, hy, T, s, A, b);
    for (int k = 0; k < 5; ++k) d[k] = 0.0;
    int top = -1, bot = -1;
    double zhi = INFINITY, zlo = -INFINITY;
    for (int i = 0; i < 14; ++i) {
        double ax = A[3 * i], ay = A[3 * i + 1], az = A[3 * i + 2];
        double rhs = b[i] - ax * u - ay * v;
        if (az > 0.0) {
            double z = rhs / az;
            if (z < zhi) { zhi = z; top = i; }
        } else if (az < 0.0) {
            double z = rhs / az;
            if (z > zlo) { zlo = z; bot = i; }
        } else if (rhs < 0.0) {
            return 0.0;
        }
    }
    if (!(zhi > zlo)) return 0.0;
    int act[2] = {top, bot};
    double sign[2] = {1.0, -1.0};
    for (int k = 0; k < 2; ++k) {
        int i = act[k];
        double ax = A[3 * i], ay = A[3 * i + 1], az = A[3 * i + 2];
        d[0] += sign[k] * (-ax / az);
        d[1] += sign[k] * (-ay / az);
        d[2] += sign[k] * db[i][0] / az;
        d[3] += sign[k] * db[i][1] / az;
        d[4] += sign[k] * db[i][2] / az;
    }
    return zhi - zlo;
}

/* Thickness of particle q at (x, y) and its gradient with respect to the
 * fields cx, cy, theta, a|hx, b|hy, T (g[0..5]; px, rad, um units of the
 * particle tensor). */
static double particle_thickness_grad(const double *q, double dx, double bevel,
                                      double x, double y, double g[6])
{
    double c = cos(q[F_TH]), s = sin(q[F_TH]);
    double ex = x - q[F_CX], ey = y - q[F_CY];
    double u = c * ex + s * ey;
    double v = -s * ex + c * ey;
    /* du/d(cx, cy, theta) and dv/d(...) */
    double du[3] = {-c, -s, v}, dv[3] = {s, -c, -u};
    for (int k = 0; k < 6; ++k) g[k] = 0.0;
    if (q[F_KIND] > 0.5) {
        double d[5];
        double t = prism_chord_grad(q[F_A] * dx, q[F_B] * dx, q[F_T], bevel, u * dx, v * dx, d);
        if (t == 0.0) return 0.0;
        for (int k = 0; k < 3; ++k) g[k] = dx * (d[0] * du[k] + d[1] * dv[k]);
        g[3] = dx * d[2];
        g[4] = dx * d[3];
        g[5] = d[4];
        return t;
    }
    double a = q[F_A], b = q[F_B];
    double r = 1.0 - (u / a) * (u / a) - (v / b) * (v / b);
    if (!(r > 0.0)) return 0.0;
    double sr = sqrt(r), t = q[F_T] * sr;
    double dtdr = q[F_T] / (2.0 * sr);
    double drdu = -2.0 * u / (a * a), drdv = -2.0 * v / (b * b);
    for (int k = 0; k < 3; ++k) g[k] = dtdr * (drdu * du[k] + drdv * dv[k]);
    g[3] = dtdr * 2.0 * u * u / (a * a * a);
    g[4] = dtdr * 2.0 * v * v / (b * b * b);
    g[5] = sr;
    return t;
}

/* d/d(defocus, shear_px, shear_angle, bias) of the transfer function of
 * one modality at DFT sample (i, j); H itself is returned in (hr, hi). */
static void transfer_grad(const orc_optics *o, int mode, int i, int j,
                          double *hr, double *hi, double dh[4][2])
{
    double kna = 2.0 * M_PI * o->NA / o->lambda;
    double k0 = 2.0 * M_PI * o->n_medium / o->lambda;
    double kx = kfreq(j, o->W, o->dx), ky = kfreq(i, o->H, o->dx);
    double qx = kx, qy = ky;
    if (mode == 2) {
        qx += o->oblique_frac * kna * cos(o->oblique_angle);
        qy += o->oblique_frac * kna * sin(o->oblique_angle);
    }
    for (int k = 0; k < 4; ++k) dh[k][0] = dh[k][1] = 0.0;
    double pr, pi;
    pupil(o, qx, qy, &pr, &pi);
    *hr = pr;
    *hi = pi;
    if (pr == 0.0 && pi == 0.0) return;
    double kappa = sqrt(k0 * k0 - qx * qx - qy * qy) - k0;  /* d chi / d dz */
    /* dP/ddz = i kappa P */
    double dpr = -kappa * pi, dpi = kappa * pr;
    if (mode != 4) {
        dh[0][0] = dpr;
        dh[0][1] = dpi;
        return;
    }
    double ca = cos(o->shear_angle), sa = sin(o->shear_angle);
    double dsx = 0.5 * o->shear_px * o->dx * ca, dsy = 0.5 * o->shear_px * o->dx * sa;
    double arg = kx * dsx + ky * dsy + o->bias_phase;
    double g = 2.0 * sin(arg), gp = 2.0 * cos(arg);
    /* H = P * i g: (pr + i pi)(i g) = (-pi g, pr g) */
    *hr = -pi * g;
    *hi = pr * g;
    dh[0][0] = -dpi * g;
    dh[0][1] = dpr * g;
    double darg[3] = {0.5 * o->dx * (kx * ca + ky * sa),
                      0.5 * o->shear_px * o->dx * (-kx * sa + ky * ca), 1.0};
    for (int k = 0; k < 3; ++k) {
        dh[k + 1][0] = -pi * gp * darg[k];
        dh[k + 1][1] = pr * gp * darg[k];
    }
}

/* Gradient of L = sum_m sum_px gI[m][px] I_m[px] (gI = dL/dI given) with
 * respect to every particle field (gsoa, [9][n] row-major, the kind row
 * zero) and to the optics scalars gopt[4] = dL/d(defocus, shear_px,
 * shear_angle, bias_phase).  Adjoint chain of orc_render:
 *   E_m = IDFT2(DFT2(E) H_m) / (HW), I_m = |E_m|^2
 *   dL/dE_m = 2 gI_m E_m; dL/dZ_m = DFT2(dL/dE_m) / (HW) with Z_m = E^ H_m;
 *   dL/dE^ = sum_m conj(H_m) dL/dZ_m; dL/dE = IDFT2(dL/dE^);
 *   dL/dOPD = (2 pi / lambda) Re(conj(dL/dE) i E), dL/dATT = -Re(conj(dL/dE) E);
 *   dL/d(dn_p) = sum t_p dL/dOPD, dL/d(mu_p) = sum t_p dL/dATT,
 *   dL/d(geometry_p) = sum (dn_p dL/dOPD + mu_p dL/dATT) dt_p/d(geometry_p);
 *   dL/d(optics) = sum_m sum_k Re(conj(dL/dZ_m) E^ dH_m/d(optics)).
 * Complex gradients are dL/dRe + i dL/dIm. */
void orc_render_grad(const float *soa, int64_t ld, int n, const orc_optics *o,
                     const double *gI, double *gsoa, double *gopt)
{
    int H = o->H, W = o->W;
    size_t hw = (size_t)H * W;
    double *opd = malloc(sizeof(double) * hw), *att = malloc(sizeof(double) * hw);
    double *er = malloc(sizeof(double) * hw), *ei = malloc(sizeof(double) * hw);
    double *fr = malloc(sizeof(double) * hw), *fi = malloc(sizeof(double) * hw);
    double *zr = malloc(sizeof(double) * hw), *zi = malloc(sizeof(double) * hw);
    double *gr = calloc(hw, sizeof(double)), *gi = calloc(hw, sizeof(double));
    double *hr = malloc(sizeof(double) * hw), *hi = malloc(sizeof(double) * hw);
    orc_opd_att(soa, ld, n, H, W, o->dx, o->bevel_slope, 0, opd, att);
    orc_field(opd, att, (int64_t)hw, o->lambda, er, ei);
    memcpy(fr, er, sizeof(double) * hw);
    memcpy(fi, ei, sizeof(double) * hw);
    orc_fft2(fr, fi, H, W, -1); /* E^ */
    for (int k = 0; k < 4; ++k) gopt[k] = 0.0;
    double inv = 1.0 / (double)hw;
    int m = 0;
    for (int bit = 0; bit < 3; ++bit) {
        int mode = 1 << bit;
        if (!(o->modes & (uint32_t)mode)) continue;
        orc_transfer(o, mode, hr, hi);
        for (size_t t = 0; t < hw; ++t) {
            zr[t] = fr[t] * hr[t] - fi[t] * hi[t];
            zi[t] = fr[t] * hi[t] + fi[t] * hr[t];
        }
        orc_fft2(zr, zi, H, W, +1); /* HW * E_m */
        const double *g = gI + (size_t)m * hw;
        for (size_t t = 0; t < hw; ++t) { /* dL/dE_m = 2 gI E_m */
            double a = zr[t] * inv, b = zi[t] * inv;
            zr[t] = 2.0 * g[t] * a;
            zi[t] = 2.0 * g[t] * b;
        }
        orc_fft2(zr, zi, H, W, -1);
        for (size_t t = 0; t < hw; ++t) { /* dL/dZ_m */
            zr[t] *= inv;
            zi[t] *= inv;
        }
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                size_t t = (size_t)i * W + j;
                double h0, h1, dh[4][2];
                transfer_grad(o, mode, i, j, &h0, &h1, dh);
                /* dL/dE^ += conj(H) dL/dZ */
                gr[t] += h0 * zr[t] + h1 * zi[t];
                gi[t] += h0 * zi[t] - h1 * zr[t];
                /* Re(conj(gZ) E^ dH) */
                for (int k = 0; k < 4; ++k) {
                    double wr = fr[t] * dh[k][0] - fi[t] * dh[k][1];
                    double wi = fr[t] * dh[k][1] + fi[t] * dh[k][0];
                    gopt[k] += zr[t] * wr + zi[t] * wi;
                }
            }
        ++m;
    }
    orc_fft2(gr, gi, H, W, +1); /* dL/dE */
    /* per-pixel dL/dOPD (into opd) and dL/dATT (into att), keeping E */
    for (size_t t = 0; t < hw; ++t) {
        double go = 2.0 * M_PI / o->lambda * (gr[t] * (-ei[t]) + gi[t] * er[t]);
        double ga = -(gr[t] * er[t] + gi[t] * ei[t]);
        opd[t] = go;
        att[t] = ga;
    }
    memset(gsoa, 0, sizeof(double) * F_COUNT * (size_t)n);
    for (int p = 0; p < n; ++p) {
        double q[F_COUNT];
        load_particle(soa, ld, p, q);
        double R = q[F_KIND] > 0.5 ? sqrt(q[F_A] * q[F_A] + q[F_B] * q[F_B]) : fmax(q[F_A], q[F_B]);
        double jl = floor(q[F_CX] - R - 1.5), jh = ceil(q[F_CX] + R + 0.5);
        double il = floor(q[F_CY] - R - 1.5), ih = ceil(q[F_CY] + R + 0.5);
        if (jh < 0 || ih < 0 || jl > W - 1 || il > H - 1) continue;
        int j0 = jl < 0 ? 0 : (int)jl, j1 = jh > W - 1 ? W - 1 : (int)jh;
        int i0 = il < 0 ? 0 : (int)il, i1 = ih > H - 1 ? H - 1 : (int)ih;
        double acc[F_COUNT] = {0};
        for (int i = i0; i <= i1; ++i)
            for (int j = j0; j <= j1; ++j) {
                double g6[6];
                double t = particle_thickness_grad(q, o->dx, o->bevel_slope, j + 0.5, i + 0.5, g6);
                if (t == 0.0) continue;
                size_t s = (size_t)i * W + j;
                double w = q[F_DN] * opd[s] + q[F_MU] * att[s];
                for (int k = 0; k < 6; ++k) acc[k] += w * g6[k];
                acc[F_DN] += t * opd[s];
                acc[F_MU] += t * att[s];
            }
        for (int f = 0; f < F_COUNT; ++f) gsoa[(size_t)f * n + p] = acc[f];
    }
    free(opd); free(att); free(er); free(ei); free(fr); free(fi);
    free(zr); free(zi); free(gr); free(gi); free(hr); free(hi);
}

/* ------------------------------------------------------------------ */
/* Sensor noise (Sec. III.C: Poisson shot plus Gaussian read noise)    */
/* ------------------------------------------------------------------ */

/* Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC 2011): ten rounds
 * of two 32x32->64-bit multiplications on a 4-word counter with a 2-word
 * key bumped by the Weyl constants between rounds. */
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0, 1) from 32 random bits. */
static double unit_open(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* The uniforms of element i, round r (four per round). */
static void noise_round(uint64_t seed, int64_t i, uint32_t r, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)(uint64_t)i, (uint32_t)((uint64_t)i >> 32), r, 0x6E6F6973u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32(ctr, key, o);
    for (int k = 0; k < 4; ++k) u[k] = unit_open(o[k]);
}

#define ORC_NOISE_ROUNDS 64

/* Poisson(lam) sample of element i: round 0 holds (u0, u1) for the normal
 * deviate and (u2, u3) for the first Poisson attempt, rounds 1.. two more
 * attempts each.
 *   lam < 10:  inversion by sequential search with u2 (pmf recursion
 *              p_k = p_{k-1} lam / k from p_0 = exp(-lam));
 *   lam >= 10: Hormann's transformed rejection with squeeze (PTRS; W.
 *              Hormann, "The transformed rejection method for generating
 *              Poisson random variables", Insurance: Mathematics and
 *              Economics 12, 1993), attempts from (u2, u3), (u4, u5), ...
 * If every attempt of ORC_NOISE_ROUNDS rounds is rejected the sample is
 * floor(lam). */
int64_t orc_poisson(double lam, uint64_t seed, int64_t i)
{
    double u[4];
    noise_round(seed, i, 0, u);
    if (!(lam > 0.0)) return 0;
    if (lam < 10.0) {
        double p = exp(-lam), F = p;
        int64_t k = 0;
        while (u[2] > F && k < 1000) {
            ++k;
            p *= lam / (double)k;
            F += p;
        }
        return k;
    }
    const double slam = sqrt(lam), loglam = log(lam);
    const double b = 0.931 + 2.53 * slam;
    const double a = -0.059 + 0.02483 * b;
    const double invalpha = 1.1239 + 1.1328 / (b - 3.4);
    const double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (uint32_t r = 0; r < ORC_NOISE_ROUNDS; ++r) {
        if (r > 0) noise_round(seed, i, r, u);
        for (int h = (r == 0 ? 1 : 0); h < 2; ++h) {
            const double U = u[2 * h] - 0.5, V = u[2 * h + 1];
            const double us = 0.5 - fabs(U);
            const double k = floor((2.0 * a / us + b) * U + lam + 0.43);
            if (us >= 0.07 && V <= vr) return (int64_t)k;
            if (k < 0.0 || (us < 0.013 && V > us)) continue;
            if (log(V * invalpha / (a / (us * us) + b)) <= -lam + k * loglam - lgamma(k + 1.0))
                return (int64_t)k;
        }
    }
    return (int64_t)floor(lam);
}

/* Standard normal deviate of element i by the Box-Muller transform of
 * round 0's (u0, u1). */
double orc_normal(uint64_t seed, int64_t i)
{
    double u[4];
    noise_round(seed, i, 0, u);
    return sqrt(-2.0 * log(u[0])) * cos(2.0 * M_PI * u[1]);
}

/* Noisy image: out_i = (Poisson(g max(I_i, 0)) + sigma Z_i) / g, with g the
 * photo-electrons per unit intensity and sigma the read noise (electrons),
 * so that the noiseless mean is I. */
void orc_sensor_noise(const float *img, int64_t count, double g, double sigma,
                      uint64_t seed, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < count; ++i) {
        double lam = g * (img[i] > 0.0f ? (double)img[i] : 0.0);
        out[i] = ((double)orc_poisson(lam, seed, i) + sigma * orc_normal(seed, i)) / g;
    }
}

/* ------------------------------------------------------------------ */
/* Image losses of inverse rendering                                   */
/* ------------------------------------------------------------------ */

/* Spectral loss of Eq. 8 (Sec. IV.B): the squared difference of the log
 * amplitude spectra of an image and a target, K images of H x W each,
 *   L = 1 / (K H W) sum_k sum_f (log(|A_k(f)| + e_k) - log(|B_k(f)| + e_k))^2,
 * A_k = F I_k and B_k = F T_k the unnormalised forward 2-D DFTs, and e_k =
 * eps_rel max_f |B_k(f)| the guard inside the logarithms (a reading: the
 * paper writes log|F(.)| with no guard; without one every frequency where
 * both spectra are only rounding noise would count as much as the band).
 * With d_f = log(|A_f| + e) - log(|B_f| + e) and A_f = a_f + i b_f,
 * dL/da_f + i dL/db_f = 2 d_f A_f / (K H W |A_f| (|A_f| + e)) (zero where
 * A_f = 0), and since A is the DFT of a real image, dL/dI = Re(G) with G the
 * unnormalised inverse DFT of that complex gradient.  grad (K H W values)
 * receives dL/dI when it is not NULL.  Returns L. */
double orc_spectral_loss(const double *img, const double *tgt, int K, int H, int W,
                         double eps_rel, double *grad)
{
    const size_t n = (size_t)H * W;
    double *ar = malloc(sizeof(double) * n), *ai = malloc(sizeof(double) * n);
    double *br = malloc(sizeof(double) * n), *bi = malloc(sizeof(double) * n);
    double total = 0.0;
    const double norm = (double)K * (double)n;
    for (int k = 0; k < K; ++k) {
        for (size_t i = 0; i < n; ++i) {
            ar[i] = img[k * n + i]; ai[i] = 0.0;
            br[i] = tgt[k * n + i]; bi[i] = 0.0;
        }
        orc_fft2(ar, ai, H, W, -1);
        orc_fft2(br, bi, H, W, -1);
        double bmax = 0.0;
        for (size_t i = 0; i < n; ++i) {
            const double m = hypot(br[i], bi[i]);
            if (m > bmax) bmax = m;
        }
        const double e = eps_rel * bmax;
        for (size_t i = 0; i < n; ++i) {
            const double ma = hypot(ar[i], ai[i]);
            const double d = log(ma + e) - log(hypot(br[i], bi[i]) + e);
            total += d * d;
            /* complex gradient, kept in (ar, ai) for the inverse transform */
            const double c = ma > 0.0 ? 2.0 * d / (norm * ma * (ma + e)) : 0.0;
            ar[i] *= c;
            ai[i] *= c;
        }
        if (grad) {
            orc_fft2(ar, ai, H, W, +1);
            for (size_t i = 0; i < n; ++i) grad[k * n + i] = ar[i];
        }
    }
    free(ar); free(ai); free(br); free(bi);
    return total / norm;
}

/* Misfit of the inverse solve's coarse-to-fine curriculum (Sec. IV.B): the
 * squared difference of the image and the target after both pass an ideal
 * low-pass filter of radius `cutoff` (cycles/um) on the frequency grid
 * f = (fftfreq(W, dx), fftfreq(H, dx)), summed over the K H W pixels and
 * multiplied by `scale`.  By Parseval this is
 *   L = scale / (H W) sum_k sum_{|f| <= cutoff} |A_k(f) - B_k(f)|^2,
 * and dL/dI = 2 scale / (H W) Re(F^-1 [m (A - B)]) with F^-1 the
 * unnormalised inverse DFT and m the filter's indicator.  grad as above. */
double orc_lowpass_misfit(const double *img, const double *tgt, int K, int H, int W,
                          double dx, double cutoff, double scale, double *grad)
{
    const size_t n = (size_t)H * W;
    double *ar = malloc(sizeof(double) * n), *ai = malloc(sizeof(double) * n);
    double total = 0.0;
    for (int k = 0; k < K; ++k) {
        for (size_t i = 0; i < n; ++i) {
            ar[i] = img[k * n + i] - tgt[k * n + i];
            ai[i] = 0.0;
        }
        orc_fft2(ar, ai, H, W, -1);  /* A - B by linearity */
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const size_t i = (size_t)y * W + x;
                const double fx = (double)(x < W / 2 ? x : x - W) / ((double)W * dx);
                const double fy = (double)(y < H / 2 ? y : y - H) / ((double)H * dx);
                if (fx * fx + fy * fy <= cutoff * cutoff) {
                    total += ar[i] * ar[i] + ai[i] * ai[i];
                } else {
                    ar[i] = 0.0;
                    ai[i] = 0.0;
                }
            }
        if (grad) {
            orc_fft2(ar, ai, H, W, +1);
            for (size_t i = 0; i < n; ++i) grad[k * n + i] = 2.0 * scale / (double)n * ar[i];
        }
    }
    free(ar); free(ai);
    return total * scale / (double)n;
}

/* Threads of the OpenMP loops above (timing on one core or all). */
#ifdef _OPENMP
#include <omp.h>
#endif
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
