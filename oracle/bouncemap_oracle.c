/*
 * Bounce-map oracle: a plain, slow FP64 CPU restatement of the discrete
 * bounce-to-bounce map of the intracavity field of a microchip laser
 * (A. Yu. Okulov, "Two-dimensional periodic and quasiperiodic spatial
 * structures in microchip laser resonator": the nonlocal map of eq.
 * conv_map, its Fresnel-kernel form eq. complex_8F with the complex aperture
 * of eq. complex_aperture2, and the operator exponent of eq.
 * limit_of_operators_renorm_final).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers.  The CUDA library
 * never links, loads or calls this file, and this file shares no code,
 * header, table or constant generator with it.
 *
 * Conventions (the readings of the paper that the map below takes):
 *   - Field E and inversion N are n x n, row-major, E[y*n + x], complex
 *     double (C99 layout: re, im interleaved).
 *   - Pixel centres: x_j = (j - n/2) / (n/2); the window half-width is 1.
 *   - Forward DFT kernel exp(-2 pi i j k / n), unnormalised.
 *   - Signed frequency index m = k for k < n/2, else k - n.
 *   - Diffraction over one iterate (eq. limit_of_operators_renorm_final,
 *     exp[i z lap / 2k] on a plane wave exp(i kappa x) gives
 *     exp(-i z kappa^2 / 2k)):
 *         E' = IDFT2( DFT2(E) * exp(-i pi alpha (mx^2 + my^2)) ) / n^2,
 *     with alpha = lambda z / W^2 = (D/W)^2 / N_F, N_F = D^2/(lambda z).
 *   - Gain slice, mirror and absorbing edge (eq. conv_map's local map f,
 *     the modulus D_0 of eq. complex_aperture2, the saturable-gain form of
 *     the class-B equations):
 *         I = |E'|^2
 *         E_{n+1} = sqrt(R) * A(x) A(y) * D(x, y) * exp(N_n / 2) * E'
 *         N_{n+1} = N_n + (N0 - N_n (1 + I / Isat)) / T1
 *     A = 0 on the outer `edge` pixels of each axis, 1 inside; with a taper
 *     of w pixels A rises inside the band as sin^2((pi/2) (d+1)/(w+1)),
 *     d = 0 .. w-1 pixels from the band (a smooth modulus D_0).
 *   - Inversion update, exact variant (relax = 1): the rate equation
 *     dN/dt = (N0 - N (1 + I/Isat)) / T1 integrated over one bounce with I
 *     held fixed, N <- Nss + (N - Nss) exp(-(1 + I/Isat)/T1),
 *     Nss = N0 / (1 + I/Isat).
 *   - Argument of the complex aperture (eq. complex_aperture2: a mirror of
 *     focal length F, phase k r^2 / 2F, and a roughness phase psi), applied
 *     complex-conjugated because the propagator above is the conjugate of
 *     the one paired with that equation (eq. Maxw_Bloch):
 *         D = exp(-i (k r^2 / (2F) + psi)),
 *     and in window units (r = x W/2, k = 2 pi/lambda, W^2/lambda = z/alpha)
 *         k r^2 / (2F) = (pi / (4 alpha)) (z / F) (x^2 + y^2).
 *     F > 0 then focuses; z/F = 0 and no psi give D = 1.
 *   - Multi-slice gain medium (the thin-slice form the integral-equation
 *     section mentions for a gain medium that is not concentrated near one
 *     plane): with m slices a bounce is m steps "diffract z/m, then slice
 *     s": E <- exp(N_s / 2) E, N_s <- N_s + (N0/m - N_s (1 + I_s/Isat))/T1
 *     with I_s = |E|^2 arriving at slice s; each slice has its own
 *     inversion and a pump of N0/m, so the small-signal gain per pass stays
 *     g0.  The mirror (sqrt R, A, D) acts once, after the last slice.  With
 *     m = 1 this is the map above.
 *   - Pump N0 = g0 * exp(-(r / r_p)^order) (super-Gaussian), g0 (uniform)
 *     or g0 * profile (array).
 *
 * Parity unpinned: the long-horizon trajectory (beyond a few tens of
 * bounces the map is chaotic; long runs are compared by statistics only).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_PI 3.14159265358979323846

/* Parameters of one resonator; mirrored field by field by the ctypes
 * structure in oracle/__init__.py. */
typedef struct {
    int n;                 /* grid side */
    double alpha;          /* lambda z / W^2 */
    double g0;             /* small-signal intensity gain exponent per pass */
    double T1;             /* inversion relaxation time, in bounces */
    double R;              /* mirror intensity reflectivity */
    double Isat;           /* saturation intensity */
    int edge;              /* absorbing edge width in pixels */
    int pump_kind;         /* 0 super-Gaussian, 1 uniform, 2 array */
    double pump_order;     /* super-Gaussian exponent */
    double pump_radius;    /* r_p as a fraction of the window half-width */
    const double *pump_profile; /* n*n values in [0,1] when pump_kind == 2 */
    double z_over_F;       /* propagation distance per bounce over the mirror's focal length (0: flat) */
    const double *roughness; /* n*n roughness phase psi in radians, or NULL */
    int slices;            /* thin gain slices per bounce (0 or 1: one) */
    int taper;             /* width of the sin^2 ramp of the aperture modulus inside the edge (0: hard) */
    int relax;             /* inversion update: 0 explicit Euler step, 1 exact over the bounce */
} orc_params;

int orc_version(void) { return 1; }

/* 1 when the library was compiled with OpenMP, so that the nthreads
 * arguments take effect; 0 when every call runs on one thread. */
int orc_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* Signed frequency of DFT bin k. */
static int signed_freq(int k, int n) { return k < n / 2 ? k : k - n; }

/* ------------------------------------------------------------------------
 * Discrete Fourier transforms (the library primitive of the split-step
 * method; eq. limit_of_operators_renorm_final is diagonal in this basis).
 * ---------------------------------------------------------------------- */

/* Brute-force DFT straight from its definition:
 * y[k] = sum_j x[j] exp(sign * 2 pi i j k / n).  The product j*k is reduced
 * modulo n in integers before the angle is formed, so the argument of cos
 * and sin stays within one turn. */
void orc_dft(const cplx *x, cplx *y, int n, int sign)
{
    for (int k = 0; k < n; ++k) {
        cplx acc = 0;
        for (int j = 0; j < n; ++j) {
            long long jk = ((long long)j * k) % n;
            double ang = sign * 2.0 * ORC_PI * (double)jk / (double)n;
            acc += x[j] * (cos(ang) + sin(ang) * _Complex_I);
        }
        y[k] = acc;
    }
}

/* Radix-2 Cooley-Tukey, decimation in time: bit-reversal reordering, then
 * log2(n) stages of butterflies.  Each twiddle is evaluated directly with
 * cos/sin (no recurrence).  Returns -1 if n is not a power of two. */
int orc_fft(cplx *x, int n, int sign)
{
    if (!is_pow2(n)) return -1;
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; ++k) {
            double ang = sign * 2.0 * ORC_PI * (double)k / (double)len;
            cplx w = cos(ang) + sin(ang) * _Complex_I;
            for (int s = 0; s < n; s += len) {
                cplx u = x[s + k];
                cplx v = x[s + k + half] * w;
                x[s + k] = u + v;
                x[s + k + half] = u - v;
            }
        }
    }
    return 0;
}

/* 2-D transform of an n x n row-major array: every row, then every column. */
int orc_fft2(cplx *a, int n, int sign, int nthreads)
{
    if (!is_pow2(n)) return -1;
    if (nthreads < 1) nthreads = 1;
    (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
    for (int y = 0; y < n; ++y) orc_fft(a + (size_t)y * n, n, sign);
#pragma omp parallel num_threads(nthreads)
    {
        cplx *col = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
        for (int x = 0; x < n; ++x) {
            for (int y = 0; y < n; ++y) col[y] = a[(size_t)y * n + x];
            orc_fft(col, n, sign);
            for (int y = 0; y < n; ++y) a[(size_t)y * n + x] = col[y];
        }
        free(col);
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Diffraction over one iterate: the paraxial transfer function
 * exp(-i pi alpha (mx^2 + my^2)) (eq. limit_of_operators_renorm_final; the
 * Fresnel kernel of eq. complex_8F in the Fourier basis).
 * ---------------------------------------------------------------------- */

/* H[ky*n + kx] = exp(-i pi alpha (mx^2 + my^2)).  The product alpha*s with
 * the integer s = mx^2 + my^2 is formed and reduced modulo 2 in long double,
 * so the phase keeps its accuracy when pi*alpha*s runs to thousands of
 * radians. */
void orc_phase_2d(int n, double alpha, cplx *H)
{
    for (int ky = 0; ky < n; ++ky) {
        long long my = signed_freq(ky, n);
        for (int kx = 0; kx < n; ++kx) {
            long long mx = signed_freq(kx, n);
            long double s = (long double)(mx * mx + my * my);
            long double t = fmodl((long double)alpha * s, 2.0L);
            double ph = -ORC_PI * (double)t;
            H[(size_t)ky * n + kx] = cos(ph) + sin(ph) * _Complex_I;
        }
    }
}

/* E <- IDFT2(DFT2(E) * H) / n^2 with a precomputed H. */
static void diffract_with(cplx *E, const cplx *H, int n, int nthreads)
{
    size_t P = (size_t)n * n;
    orc_fft2(E, n, -1, nthreads);
    for (size_t i = 0; i < P; ++i) E[i] *= H[i];
    orc_fft2(E, n, +1, nthreads);
    double inv = 1.0 / (double)P;
    for (size_t i = 0; i < P; ++i) E[i] *= inv;
}

int orc_diffract(cplx *E, int n, double alpha, int nthreads)
{
    if (!is_pow2(n)) return -1;
    cplx *H = (cplx *)malloc(sizeof(cplx) * (size_t)n * n);
    if (!H) return -2;
    orc_phase_2d(n, alpha, H);
    diffract_with(E, H, n, nthreads);
    free(H);
    return 0;
}

/* ------------------------------------------------------------------------
 * Pump, i.e. the unsaturated inversion N0(x, y).
 * ---------------------------------------------------------------------- */

static double pixel_coord(int j, int n) { return (double)(j - n / 2) / (double)(n / 2); }

void orc_pump(const orc_params *p, double *N0)
{
    int n = p->n;
    for (int y = 0; y < n; ++y) {
        for (int x = 0; x < n; ++x) {
            double v;
            if (p->pump_kind == 1) {
                v = p->g0;
            } else if (p->pump_kind == 2) {
                v = p->g0 * p->pump_profile[(size_t)y * n + x];
            } else {
                double xr = pixel_coord(x, n), yr = pixel_coord(y, n);
                double r = sqrt(xr * xr + yr * yr);
                v = p->g0 * exp(-pow(r / p->pump_radius, p->pump_order));
            }
            N0[(size_t)y * n + x] = v;
        }
    }
}

/* ------------------------------------------------------------------------
 * Seeded initial noise: splitmix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator, then the Box-Muller transform.
 * ---------------------------------------------------------------------- */

/* The c-th output (c = 0, 1, ...) of a splitmix64 stream whose state starts
 * at `seed`: the state after c+1 increments of the golden gamma, passed
 * through the splitmix64 finaliser. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* E[i] = sigma * sqrt(-2 ln(1 - u1)) * exp(2 pi i u2), sigma = amp / sqrt(2),
 * with u1, u2 the top 53 bits of outputs 2i and 2i+1 scaled to [0, 1).
 * Each of Re and Im is then normal with variance amp^2 / 2, so
 * E|E|^2 = amp^2. */
void orc_noise(int n, uint64_t seed, double amp, cplx *E)
{
    size_t P = (size_t)n * n;
    double sigma = amp / sqrt(2.0);
    for (size_t i = 0; i < P; ++i) {
        double u1 = (double)(orc_splitmix64(seed, 2 * (uint64_t)i) >> 11) * 0x1.0p-53;
        double u2 = (double)(orc_splitmix64(seed, 2 * (uint64_t)i + 1) >> 11) * 0x1.0p-53;
        double rho = sigma * sqrt(-2.0 * log(1.0 - u1));
        double th = 2.0 * ORC_PI * u2;
        E[i] = rho * cos(th) + rho * sin(th) * _Complex_I;
    }
}

/* ------------------------------------------------------------------------
 * Structured starting fields: the Gaussian beam, the periodic array of
 * Gaussian beams and the array of first-order vortices of the exact
 * solutions (eqs. Field_exact11, Field_exact112), on the periodic window.
 * ---------------------------------------------------------------------- */

/* Mirrored field by field by the ctypes structure in oracle/__init__.py. */
typedef struct {
    int kind;            /* 0 Gaussian beam, 1 array of Gaussian beams, 2 array of vortices */
    int periods;         /* q lattice periods across the window (period p = 2/q) */
    int out_of_phase;    /* alternate neighbours: beam sign (kind 1) or vortex charge (kind 2) */
    double width;        /* Gaussian radius w of a beam or vortex core */
    double envelope;     /* radius of the common Gaussian envelope (0: none) */
    double curvature;    /* common phase front exp(-i c r^2) */
    double amplitude;
} orc_pattern_t;

static double pixel_coord_of(int j, int n) { return (double)(j - n / 2) / (double)(n / 2); }

/* Shortest signed displacement on the periodic window of width 2. */
static double wrap2(double u) { return u - 2.0 * floor(u / 2.0 + 0.5); }

/* E(x, y) = amplitude * exp(-r^2 / (2 envelope^2)) * exp(-i c r^2) * S(x, y)
 * with S = exp(-r^2/(2w^2)) for the single beam, and for the arrays the sum
 * over the q*q lattice points (a p, b p), a, b = 0..q-1, of
 *   beams:    s_ab exp(-d^2/(2w^2)),                 s_ab = (-1)^(a+b) or 1
 *   vortices: ((dx + i k_ab dy)/w) exp(-d^2/(2w^2)),  k_ab = (-1)^(a+b) or 1
 * (k_ab the topological charge), with (dx, dy) the shortest displacement
 * from the lattice point on the periodic window; points whose Gaussian
 * exponent d^2/(2w^2) exceeds 50 are left out.  Returns -1 on bad input. */
int orc_pattern(int n, const orc_pattern_t *pt, cplx *E)
{
    if (!is_pow2(n) || pt->width <= 0.0 || pt->envelope < 0.0 || pt->kind < 0 || pt->kind > 2) return -1;
    if (pt->kind > 0 && (pt->periods < 1 || (pt->out_of_phase && pt->periods % 2))) return -1;
    int q = pt->periods;
    double p = 2.0 / (double)q, w2 = pt->width * pt->width;
    for (int y = 0; y < n; ++y) {
        double yc = pixel_coord_of(y, n);
        for (int x = 0; x < n; ++x) {
            double xc = pixel_coord_of(x, n);
            double r2 = xc * xc + yc * yc;
            cplx S = 0.0;
            if (pt->kind == 0) {
                S = exp(-r2 / (2.0 * w2));
            } else {
                for (int b = 0; b < q; ++b) {
                    double dy = wrap2(yc - b * p);
                    for (int a = 0; a < q; ++a) {
                        double dx = wrap2(xc - a * p);
                        double e = (dx * dx + dy * dy) / (2.0 * w2);
                        if (e > 50.0) continue;
                        double alt = pt->out_of_phase && ((a + b) & 1) ? -1.0 : 1.0;
                        if (pt->kind == 1)
                            S += alt * exp(-e);
                        else
                            S += (dx + alt * dy * _Complex_I) / pt->width * exp(-e);
                    }
                }
            }
            double env = pt->envelope > 0.0 ? exp(-r2 / (2.0 * pt->envelope * pt->envelope)) : 1.0;
            double ph = -pt->curvature * r2;
            E[(size_t)y * n + x] = pt->amplitude * env * (cos(ph) + sin(ph) * _Complex_I) * S;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * The bounce map.
 * ---------------------------------------------------------------------- */

static int inside_edge(int j, int n, int edge) { return j >= edge && j < n - edge; }

/* Aperture modulus along one axis (hard edge, optional sin^2 taper). */
static double edge_modulus(int j, int n, int edge, int taper)
{
    if (!inside_edge(j, n, edge)) return 0.0;
    int d = j - edge < n - 1 - edge - j ? j - edge : n - 1 - edge - j;
    if (d >= taper) return 1.0;
    double s = sin(0.5 * ORC_PI * (double)(d + 1) / (double)(taper + 1));
    return s * s;
}

/* Argument k r^2/(2F) + psi of the complex aperture at pixel (x, y), in
 * window units (see the conventions above). */
static double aperture_argument(const orc_params *p, int x, int y)
{
    int n = p->n;
    double xc = (double)(x - n / 2) / (double)(n / 2);
    double yc = (double)(y - n / 2) / (double)(n / 2);
    double theta = ORC_PI / (4.0 * p->alpha) * p->z_over_F * (xc * xc + yc * yc);
    if (p->roughness) theta += p->roughness[(size_t)y * n + x];
    return theta;
}

/* Local part of the map (eq. conv_map's f, the mirror and the complex
 * aperture D_0 exp(-i theta)): gain against the frozen inversion N_n, then
 * relaxation of N toward the pump driven by the arriving intensity |E'|^2.
 * One slice of m: pump N0/m; the mirror only when `mirror` is set. */
static void gain_step(cplx *E, double *N, const double *N0, const orc_params *p, int m, int mirror)
{
    int n = p->n;
    double sqrtR = mirror ? sqrt(p->R) : 1.0;
    int phased = mirror && (p->z_over_F != 0.0 || p->roughness != NULL);
    for (int y = 0; y < n; ++y) {
        for (int x = 0; x < n; ++x) {
            size_t i = (size_t)y * n + x;
            double inten = creal(E[i]) * creal(E[i]) + cimag(E[i]) * cimag(E[i]);
            double Nn = N[i];
            double A = mirror ? edge_modulus(x, n, p->edge, p->taper) * edge_modulus(y, n, p->edge, p->taper) : 1.0;
            cplx D = A;
            if (phased) {
                double theta = aperture_argument(p, x, y);
                D = A * (cos(theta) - sin(theta) * _Complex_I);
            }
            E[i] = sqrtR * exp(0.5 * Nn) * D * E[i];
            double a = 1.0 + inten / p->Isat;
            double pump = N0[i] / (double)m;
            if (p->relax) {
                double Nss = pump / a;
                N[i] = Nss + (Nn - Nss) * exp(-a / p->T1);
            } else {
                N[i] = Nn + (pump - Nn * a) / p->T1;
            }
        }
    }
}

static double mean_intensity(const cplx *E, size_t P)
{
    double s = 0.0;
    for (size_t i = 0; i < P; ++i) s += creal(E[i]) * creal(E[i]) + cimag(E[i]) * cimag(E[i]);
    return s / (double)P;
}

/* Run nb bounces in place on (E, N); N holds one n*n inversion per slice
 * (slice-major).  hist (may be NULL) receives the mean intensity
 * <|E_{b+1}|^2> after each bounce b = 0 .. nb-1.
 * Returns 0, or -1 on invalid parameters, -2 on allocation failure. */
int orc_run(const orc_params *p, cplx *E, double *N, long long nb, double *hist, int nthreads)
{
    int n = p->n;
    int m = p->slices > 1 ? p->slices : 1;
    if (!is_pow2(n) || p->T1 <= 0.0 || p->R < 0.0 || p->Isat <= 0.0 || p->edge < 0 || p->slices < 0) return -1;
    if (p->pump_kind == 2 && !p->pump_profile) return -1;
    size_t P = (size_t)n * n;
    cplx *H = (cplx *)malloc(sizeof(cplx) * P);
    double *N0 = (double *)malloc(sizeof(double) * P);
    if (!H || !N0) { free(H); free(N0); return -2; }
    orc_phase_2d(n, p->alpha / (double)m, H);
    orc_pump(p, N0);
    for (long long b = 0; b < nb; ++b) {
        for (int s = 0; s < m; ++s) {
            diffract_with(E, H, n, nthreads);
            gain_step(E, N + (size_t)s * P, N0, p, m, s == m - 1);
        }
        if (hist) hist[b] = mean_intensity(E, P);
    }
    free(H);
    free(N0);
    return 0;
}

/* ------------------------------------------------------------------------
 * Reporting: the far-field spectrum and its dominant spatial frequency.
 * ---------------------------------------------------------------------- */

/* S = |DFT2(E)|^2 (unnormalised). */
int orc_spectrum(const cplx *E, int n, double *S, int nthreads)
{
    if (!is_pow2(n)) return -1;
    size_t P = (size_t)n * n;
    cplx *T = (cplx *)malloc(sizeof(cplx) * P);
    if (!T) return -2;
    memcpy(T, E, sizeof(cplx) * P);
    orc_fft2(T, n, -1, nthreads);
    for (size_t i = 0; i < P; ++i) S[i] = creal(T[i]) * creal(T[i]) + cimag(T[i]) * cimag(T[i]);
    free(T);
    return 0;
}

/* Dominant spatial frequency, with m and -m taken as one peak: bin k and its
 * mirror k' = (-ky mod n, -kx mod n) carry the folded power S[k] + S[k']
 * (S[k] alone when k' == k), filed under the smaller flat index.  With
 * ring > 0 only bins with max(|mx|, |my|) >= ring compete.  Ties go to the
 * smaller flat index.  Writes the signed (mx, my) of the winner, its folded
 * power, and the largest folded power of any other bin. */
void orc_spectrum_peak(const double *S, int n, int ring, int *mx_out, int *my_out,
                       double *peak_out, double *runner_up_out)
{
    double best = -1.0, second = -1.0;
    long long best_k = -1;
    for (int ky = 0; ky < n; ++ky) {
        for (int kx = 0; kx < n; ++kx) {
            long long k = (long long)ky * n + kx;
            long long kp = (long long)((n - ky) % n) * n + (n - kx) % n;
            if (kp < k) continue;
            int mx = signed_freq(kx, n), my = signed_freq(ky, n);
            int amx = mx < 0 ? -mx : mx, amy = my < 0 ? -my : my;
            int cheb = amx > amy ? amx : amy;
            if (cheb < ring) continue;
            double v = (kp == k) ? S[k] : S[k] + S[kp];
            if (v > best) {
                second = best;
                best = v;
                best_k = k;
            } else if (v > second) {
                second = v;
            }
        }
    }
    if (best_k < 0) {
        *mx_out = 0; *my_out = 0; *peak_out = 0.0; *runner_up_out = 0.0;
        return;
    }
    *mx_out = signed_freq((int)(best_k % n), n);
    *my_out = signed_freq((int)(best_k / n), n);
    *peak_out = best;
    *runner_up_out = second < 0.0 ? 0.0 : second;
}
