/*
 * FP64 CPU oracle for synthetic-aperture-sonar time-domain backprojection.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * Every routine evaluates its definition directly in double precision:
 * no tables, no blocking, no differential-range tricks.  Pixels (or pings) are
 * distributed over OpenMP threads; each output element is summed by exactly
 * one thread in a fixed order, so results do not depend on the thread count.
 *
 * Paper: "GPU Acceleration for Synthetic Aperture Sonar Image Reconstruction"
 * (ASASIN), arXiv 2101.05888.
 *   Eq. 1  forward model e(t, x_RX) = int sigma(x) q(t - (|x_TX-x|+|x_RX-x|)/c) / (...) dx
 *   Sec. II-A  backprojection inverts Eq. 1 independently for every pixel
 *   Eq. 2  attitude rotation p~ = R(roll, pitch, yaw) p, NED frame (Sec. II-B)
 *
 * Parity status of each routine (what pins it) is listed above the routine.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: attitude matrix, entries exactly as printed in the paper.
 * roll = phi, pitch = theta, yaw = psi, radians.  Row-major R[3][3].
 * Pinned by: orthonormality, det = +1, the sign conventions stated under
 * Eq. 2 (positive roll lowers starboard, positive pitch raises the bow,
 * positive yaw turns to starboard), and equality with the product of the
 * three textbook single-axis rotations Rz(yaw) Ry(pitch) Rx(roll).        */
void oracle_attitude_matrix(double roll, double pitch, double yaw, double R[9]) {
    const double cph = cos(roll), sph = sin(roll);
    const double cth = cos(pitch), sth = sin(pitch);
    const double cps = cos(yaw), sps = sin(yaw);
    R[0] = cth * cps;
    R[1] = cps * sth * sph - cph * sps;
    R[2] = cph * cps * sth + sph * sps;
    R[3] = cth * sps;
    R[4] = cph * cps + sth * sph * sps;
    R[5] = cph * sth * sps - cps * sph;
    R[6] = -sth;
    R[7] = cth * sph;
    R[8] = cth * cph;
}

/* Transmitter and receiver positions per ping (Sec. II-C: attitude and lever
 * arms Omega_i place the transducers relative to the vehicle position p_i):
 *   x_TX,i   = p_i + dp_i + R_i l_TX
 *   x_RX,i,c = p_i + dp_i + R_i l_c
 * dp_i is an optional per-ping position offset (NULL = zero), the variable the
 * autofocus gradient is taken against.  Stop-and-hop: one position per ping.
 * Pinned by: zero attitude reduces to p + l; pure yaw rotates the lever in the
 * horizontal plane; the brute-force restatement in brute.py.              */
void oracle_sensor_positions(int P, int C, const double* pos, const double* att,
                             const double* tx_lever, const double* rx_lever,
                             const double* offsets, double* tx, double* rx) {
    for (int i = 0; i < P; ++i) {
        double R[9];
        oracle_attitude_matrix(att[3 * i + 0], att[3 * i + 1], att[3 * i + 2], R);
        double base[3];
        for (int a = 0; a < 3; ++a) base[a] = pos[3 * i + a] + (offsets ? offsets[3 * i + a] : 0.0);
        for (int a = 0; a < 3; ++a)
            tx[3 * i + a] = base[a] + R[3 * a + 0] * tx_lever[0] + R[3 * a + 1] * tx_lever[1] +
                            R[3 * a + 2] * tx_lever[2];
        for (int c = 0; c < C; ++c) {
            const double* l = rx_lever + 3 * c;
            double* o = rx + 3 * ((size_t)i * C + c);
            for (int a = 0; a < 3; ++a)
                o[a] = base[a] + R[3 * a + 0] * l[0] + R[3 * a + 1] * l[1] + R[3 * a + 2] * l[2];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Modified Bessel functions from their power series (Abramowitz & Stegun
 * 9.6.10):  I0(x) = sum_m ((x/2)^m / m!)^2,
 *           I1(x)/x = (1/2) sum_m (x/2)^(2m) / (m! (m+1)!).
 * Summed until the term falls below 1e-17 of the partial sum.
 * Pinned by: scipy.special.i0 / i1.                                        */
double oracle_bessel_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int m = 1; m < 500; ++m) {
        term *= q / ((double)m * (double)m);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

double oracle_bessel_i1_over_x(double x) {
    const double q = 0.25 * x * x;
    double term = 0.5, sum = 0.5;
    for (int m = 1; m < 500; ++m) {
        term *= q / ((double)m * (double)(m + 1));
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

/* ------------------------------------------------------------------------ */
/* Interpolation weights.  The paper does not state its interpolator; this
 * build reads it as a Kaiser-windowed sinc of N taps normalised to unit sum:
 *   v(d) = sinc(d) * I0(beta sqrt(1 - (d/h)^2)) / I0(beta),  |d| < h = N/2,
 *   w_m(f) = v(f - k_m) / sum_m' v(f - k_m'),   k_m = m - N/2 + 1,
 * where f in [0,1) is the fractional sample position and k_m the tap offset
 * from floor(u).  dw (optional) is dw_m/df, from the closed-form derivatives
 *   sinc'(d) = (pi d cos(pi d) - sin(pi d)) / (pi d^2),
 *   W'(d)    = -(beta^2 d / h^2) * [I1(beta s)/(beta s)] / I0(beta),  s = sqrt(1-(d/h)^2).
 * Pinned by: f = 0 gives a unit impulse; unit sum; mirror symmetry
 * w_m(f) = w_{N-1-m}(1-f); continuity w(f->1) = w(0) shifted by one tap;
 * band-limited tone error bounds; dw against central differences;
 * the scipy-based restatement in brute.py.                                 */
static double sinc_pi(double d) {
    if (d == 0.0) return 1.0;
    const double x = ORACLE_PI * d;
    return sin(x) / x;
}

static double sinc_pi_deriv(double d) {
    if (d == 0.0) return 0.0;
    const double x = ORACLE_PI * d;
    return (x * cos(x) - sin(x)) / (ORACLE_PI * d * d);
}

void oracle_kaiser_sinc_weights(double f, int taps, double beta, double* w, double* dw) {
    const double h = 0.5 * taps;
    const double i0b = oracle_bessel_i0(beta);
    double v[64], dv[64];
    double vs = 0.0, dvs = 0.0;
    for (int m = 0; m < taps; ++m) {
        const double k = (double)(m - taps / 2 + 1);
        const double d = f - k;
        double val = 0.0, der = 0.0;
        if (fabs(d) < h) {
            const double s2 = 1.0 - (d / h) * (d / h);
            const double s = sqrt(s2);
            const double win = oracle_bessel_i0(beta * s) / i0b;
            const double dwin = -(beta * beta * d / (h * h)) * oracle_bessel_i1_over_x(beta * s) / i0b;
            val = sinc_pi(d) * win;
            der = sinc_pi_deriv(d) * win + sinc_pi(d) * dwin;
        }
        v[m] = val;
        dv[m] = der;
        vs += val;
        dvs += der;
    }
    for (int m = 0; m < taps; ++m) {
        w[m] = v[m] / vs;
        if (dw) dw[m] = (dv[m] * vs - v[m] * dvs) / (vs * vs);
    }
}

/* ------------------------------------------------------------------------ */
/* Shared per-(pixel, ping, channel) evaluation of the backprojection term.
 * Two-way delay (Eq. 1 argument of q):  tau = (|x - x_TX| + |x - x_RX|) / c.
 * Fractional sample position u = (tau - t0) fs; taps j = floor(u) + k_m,
 * echo samples outside [0, Ns) read as zero.                               */
typedef struct {
    double tau, u, f;
    long j0;
    double rt, rr;           /* one-way ranges (receiver: at the time of reception) */
    double ut[3], ur[3];     /* unit vectors sensor -> pixel */
    double kappa;            /* c / (c + ur . v): dtau/d(dp) = -(ut + ur) kappa / c */
} oracle_delay;

/* Sediment-water interface (Sec. III-B: a refraction model in the
 * propagation time for sub-bottom imaging).  This build's reading: a flat
 * interface at z = g_zint (NED, z down), water above with the signal's sound
 * speed c, sediment below with speed g_csed.  A leg from a sensor s in the
 * water to a point x below the interface crosses it at the point P that
 * makes the travel time |P - s|/c + |x - P|/c_sed stationary (Fermat), so
 * its length in water metres is L = |P - s| + (c/c_sed) |x - P|; legs to
 * points at or above the interface, or from sensors at or below it, are
 * straight.  g_csed <= 0 switches the model off (the default).  Set by
 * oracle_set_medium; read by every delay evaluation.
 * Pinned by: c_sed = c gives the straight leg; a vertical leg has the
 * closed form a + (c/c_sed) b; the bisection root against a bounded scalar
 * minimiser of L (scipy); a point below the interface focuses to A P C only
 * with the model.                                                          */
static double g_zint = 0.0, g_csed = 0.0;

void oracle_set_medium(double z_interface, double c_sediment) {
    g_zint = z_interface;
    g_csed = c_sediment;
}

/* One leg sensor s -> point x: length in water metres and the unit vector
 * of its water part (from s; dL/ds = -u).                                  */
static double leg_eval(const double* x, const double* s, double c, double* u) {
    const double d0 = x[0] - s[0], d1 = x[1] - s[1], d2 = x[2] - s[2];
    if (!(g_csed > 0.0) || x[2] <= g_zint || s[2] >= g_zint) {
        const double L = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        u[0] = d0 / L;
        u[1] = d1 / L;
        u[2] = d2 / L;
        return L;
    }
    const double n = c / g_csed;
    const double a = g_zint - s[2], b = x[2] - g_zint;
    const double rho = sqrt(d0 * d0 + d1 * d1);
    /* horizontal distance xi of the crossing point from s: the root of
     * xi / sqrt(xi^2 + a^2) - n (rho - xi) / sqrt((rho - xi)^2 + b^2), which
     * increases from <= 0 at xi = 0 to >= 0 at xi = rho (bisection)        */
    double lo = 0.0, hi = rho;
    for (int it = 0; it < 200 && hi - lo > 1e-16 * (rho + a + b); ++it) {
        const double m = 0.5 * (lo + hi);
        const double f = m / sqrt(m * m + a * a) - n * (rho - m) / sqrt((rho - m) * (rho - m) + b * b);
        if (f > 0.0) hi = m;
        else lo = m;
    }
    const double xi = 0.5 * (lo + hi);
    const double w0 = rho > 0.0 ? xi * d0 / rho : 0.0, w1 = rho > 0.0 ? xi * d1 / rho : 0.0, w2 = a;
    const double lw = sqrt(w0 * w0 + w1 * w1 + w2 * w2);
    u[0] = w0 / lw;
    u[1] = w1 / lw;
    u[2] = w2 / lw;
    return lw + n * sqrt((rho - xi) * (rho - xi) + b * b);
}

/* Two-way delay of pixel x for transmitter t and receiver r (Sec. II-A).
 * v == NULL: stop-and-hop, tau = (|x - t| + |x - r|) / c.
 * v != NULL: the transmitter sends at time 0 from t and the receiver moves
 * on during reception, r(t') = r + v t' (the motion model of Sec. II-D,
 * transmission instantaneous): tau solves c tau = |x - t| + |x - r - v tau|,
 * found by fixed-point iteration (a contraction with factor |v|/c) until
 * the update is below 1e-15 tau.                                          */
static void delay_eval(const double* x, const double* t, const double* r, const double* v, double c,
                       double t0, double fs, oracle_delay* o) {
    double dt[3], dr[3];
    for (int a = 0; a < 3; ++a) {
        dt[a] = x[a] - t[a];
        dr[a] = x[a] - r[a];
    }
    o->kappa = 1.0;
    if (g_csed > 0.0) {
        /* refraction model (stop-and-hop only) */
        if (v) {
            o->tau = 0.0 / 0.0;
            return;
        }
        o->rt = leg_eval(x, t, c, o->ut);
        o->rr = leg_eval(x, r, c, o->ur);
        o->tau = (o->rt + o->rr) / c;
        o->u = (o->tau - t0) * fs;
        const double fl0 = floor(o->u);
        o->j0 = (long)fl0;
        o->f = o->u - fl0;
        return;
    }
    o->rt = sqrt(dt[0] * dt[0] + dt[1] * dt[1] + dt[2] * dt[2]);
    o->rr = sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
    o->tau = (o->rt + o->rr) / c;
    if (v) {
        for (int it = 0; it < 100; ++it) {
            double w[3];
            for (int a = 0; a < 3; ++a) w[a] = dr[a] - v[a] * o->tau;
            const double rr = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            const double tau = (o->rt + rr) / c;
            const double step = fabs(tau - o->tau);
            o->tau = tau;
            o->rr = rr;
            if (step <= 1e-15 * tau) break;
        }
        for (int a = 0; a < 3; ++a) dr[a] -= v[a] * o->tau;
        o->rr = sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
    }
    for (int a = 0; a < 3; ++a) {
        o->ut[a] = dt[a] / o->rt;
        o->ur[a] = dr[a] / o->rr;
    }
    if (v) o->kappa = c / (c + o->ur[0] * v[0] + o->ur[1] * v[1] + o->ur[2] * v[2]);
    o->u = (o->tau - t0) * fs;
    const double fl = floor(o->u);
    o->j0 = (long)fl;
    o->f = o->u - fl;
}

/* Exported for tests: tau and kappa of delay_eval (v may be NULL). */
void oracle_delay_eval(const double* x, const double* t, const double* r, const double* v, double c, double* out2) {
    oracle_delay d;
    delay_eval(x, t, r, v, c, 0.0, 1.0, &d);
    out2[0] = d.tau;
    out2[1] = d.kappa;
}

/* Beam field of view (Sec. II-C: each pixel is tested against the
 * transmit and receive beams).  This build's reading: every transducer has
 * an azimuth beam of full width theta centred on the vehicle's side axis
 * (body +y for side = +1, starboard; -y for side = -1, port), elevation
 * unrestricted.  Sensor s of ping i sees x iff b = R_i^T (x - x_s) satisfies
 * side * b_y > 0 and |b_x| <= tan(theta/2) * side * b_y.  A (ping, channel)
 * term counts iff the transmitter and that receiver both see x.
 * beam_tan = tan(theta/2) <= 0 switches the test off.
 * Pinned by: the NumPy restatement (arctan2 of body-frame vectors) in
 * brute.py, and beam off = unmasked sum.                                  */
static int sensor_sees(const double* R, const double* x, const double* s, double beam_tan, int side) {
    const double v0 = x[0] - s[0], v1 = x[1] - s[1], v2 = x[2] - s[2];
    const double bx = R[0] * v0 + R[3] * v1 + R[6] * v2;   /* R^T v, row 0 = column 0 of R */
    const double by = (R[1] * v0 + R[4] * v1 + R[7] * v2) * (double)side;
    return by > 0.0 && fabs(bx) <= beam_tan * by;
}

/* One term of the backprojection sum: pixel x, ping i, channel ch
 * (Sec. II-A): s = sum_m w_m(f) e[i][ch][j0 + k_m] (zero outside the row)
 * rotated by exp(+j 2 pi fc tau).  w: scratch of at least taps doubles.      */
static void term_eval(const double* x, int i, int ch, int C, const double* tx, const double* rx,
                      const double* vel, double fc, double fs, double c, double t0, int Ns, const void* echo,
                      int echo_f32, int taps, double beta, double* w, double* tre, double* tim) {
    oracle_delay d;
    delay_eval(x, tx + 3 * i, rx + 3 * ((size_t)i * C + ch), vel ? vel + 3 * i : NULL, c, t0, fs, &d);
    oracle_kaiser_sinc_weights(d.f, taps, beta, w, NULL);
    const size_t row = 2 * ((size_t)i * C + ch) * (size_t)Ns;
    double sr = 0.0, si = 0.0;
    for (int m = 0; m < taps; ++m) {
        const long j = d.j0 + (m - taps / 2 + 1);
        if (j < 0 || j >= Ns) continue;
        /* complex64 input is widened exactly to FP64 */
        const double er = echo_f32 ? (double)((const float*)echo)[row + 2 * j] : ((const double*)echo)[row + 2 * j];
        const double ei = echo_f32 ? (double)((const float*)echo)[row + 2 * j + 1]
                                   : ((const double*)echo)[row + 2 * j + 1];
        sr += w[m] * er;
        si += w[m] * ei;
    }
    double ph = fc * d.tau;
    ph -= floor(ph);
    const double cs = cos(2.0 * ORACLE_PI * ph), sn = sin(2.0 * ORACLE_PI * ph);
    *tre = sr * cs - si * sn;
    *tim = sr * sn + si * cs;
}

/* Backprojection (Sec. II-A, Eq. 1 inverted per pixel; pixels independent):
 *   I(x) = sum_i sum_c sum_m w_m(f) e[i][c][j0 + k_m] exp(+j 2 pi fc tau_ic(x))
 * echo: [P][C][Ns] complex interleaved (re, im), FP64 or (echo_f32 = 1) FP32;
 * pix: [npix][3]; out: [npix][2].  att [P][3] (roll, pitch, yaw) with
 * beam_tan > 0 applies the beam field of view (see sensor_sees).
 * Pinned by: NumPy brute force (brute.py) to 1e-12; linearity in the echo;
 * translation invariance; closed-form point-scatterer response (peak at the
 * scatterer, |I| = A P C within the interpolator error, phase = arg A).    */
void oracle_backproject(int P, int C, const double* tx, const double* rx, double fc, double fs,
                        double c, double t0, int Ns, const void* echo, int echo_f32, int taps,
                        double beta, long npix, const double* pix, double* out,
                        const double* att, double beam_tan, int side, const double* vel, int nthreads) {
    set_threads(nthreads);
    const int beam = att != NULL && beam_tan > 0.0;
#pragma omp parallel for schedule(dynamic, 8)
    for (long p = 0; p < npix; ++p) {
        const double* x = pix + 3 * p;
        double acc_re = 0.0, acc_im = 0.0;
        double w[64];
        for (int i = 0; i < P; ++i) {
            double R[9];
            if (beam) {
                oracle_attitude_matrix(att[3 * i], att[3 * i + 1], att[3 * i + 2], R);
                if (!sensor_sees(R, x, tx + 3 * i, beam_tan, side)) continue;
            }
            for (int ch = 0; ch < C; ++ch) {
                if (beam && !sensor_sees(R, x, rx + 3 * ((size_t)i * C + ch), beam_tan, side)) continue;
                double tre, tim;
                term_eval(x, i, ch, C, tx, rx, vel, fc, fs, c, t0, Ns, echo, echo_f32, taps, beta, w, &tre, &tim);
                acc_re += tre;
                acc_im += tim;
            }
        }
        out[2 * p] = acc_re;
        out[2 * p + 1] = acc_im;
    }
}

/* Beam decision of one sensor with a relative margin eps: +1 when the
 * decision "sees" of sensor_sees holds with both of its inequalities
 * satisfied by more than eps |b| (distances in the (b_x, b_y) plane), -1 when
 * one of them fails by more than eps |b|, 0 otherwise (the decision could
 * flip under a relative perturbation of the geometry of order eps).        */
static int sensor_class(const double* R, const double* x, const double* s, double beam_tan, int side,
                        double eps) {
    const double v0 = x[0] - s[0], v1 = x[1] - s[1], v2 = x[2] - s[2];
    const double bx = R[0] * v0 + R[3] * v1 + R[6] * v2;
    const double by = (R[1] * v0 + R[4] * v1 + R[7] * v2) * (double)side;
    const double nb = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    const double m1 = by / nb;
    const double m2 = (beam_tan * by - fabs(bx)) / (sqrt(1.0 + beam_tan * beam_tan) * nb);
    if (m1 > eps && m2 > eps) return 1;
    if (m1 < -eps || m2 < -eps) return -1;
    return 0;
}

/* Backprojection with the beam field of view split by decision margin:
 * out_sure [npix][2] sums the terms whose transmitter and receiver both see
 * the pixel by more than eps (relative), amb [npix] sums |term| over the
 * terms whose decision is within eps of flipping (neither surely in nor
 * surely out).  Any evaluation of the beam test whose relative error is
 * below eps gives sum(out_sure) + a subset of the ambiguous terms, so
 * |I - out_sure| <= amb pixel by pixel.  Requires att and beam_tan > 0.
 * Pinned by: NumPy restatement of the margins (brute.py); eps -> 0 gives
 * oracle_backproject and amb = 0.                                          */
void oracle_backproject_beam_split(int P, int C, const double* tx, const double* rx, double fc, double fs,
                                   double c, double t0, int Ns, const void* echo, int echo_f32, int taps,
                                   double beta, long npix, const double* pix, const double* att,
                                   double beam_tan, int side, double eps, double* out_sure, double* amb,
                                   const double* vel, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
    for (long p = 0; p < npix; ++p) {
        const double* x = pix + 3 * p;
        double acc_re = 0.0, acc_im = 0.0, acc_amb = 0.0;
        double w[64];
        for (int i = 0; i < P; ++i) {
            double R[9];
            oracle_attitude_matrix(att[3 * i], att[3 * i + 1], att[3 * i + 2], R);
            const int kt = sensor_class(R, x, tx + 3 * i, beam_tan, side, eps);
            if (kt < 0) continue;
            for (int ch = 0; ch < C; ++ch) {
                const int kr = sensor_class(R, x, rx + 3 * ((size_t)i * C + ch), beam_tan, side, eps);
                if (kr < 0) continue;
                double tre, tim;
                term_eval(x, i, ch, C, tx, rx, vel, fc, fs, c, t0, Ns, echo, echo_f32, taps, beta, w, &tre, &tim);
                if (kt > 0 && kr > 0) {
                    acc_re += tre;
                    acc_im += tim;
                } else {
                    acc_amb += sqrt(tre * tre + tim * tim);
                }
            }
        }
        out_sure[2 * p] = acc_re;
        out_sure[2 * p + 1] = acc_im;
        amb[p] = acc_amb;
    }
}

/* Linear adjoint of oracle_backproject (image -> echo):
 *   e_adj[i][c][j0 + k_m] += w_m(f) exp(-j 2 pi fc tau_ic(x)) I(x)
 * summed over the given pixels; echo_adj [P][C][Ns][2] is overwritten.
 * One thread owns one (ping, channel) row, so there are no races.
 * Pinned by: the dot-product test <B e, I> = <e, B^H I> in FP64.          */
void oracle_backproject_adjoint(int P, int C, const double* tx, const double* rx, double fc,
                                double fs, double c, double t0, int Ns, int taps, double beta,
                                long npix, const double* pix, const double* img, double* echo_adj,
                                const double* att, double beam_tan, int side, const double* vel, int nthreads) {
    set_threads(nthreads);
    const long rows = (long)P * C;
    const int beam = att != NULL && beam_tan > 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < rows; ++r) {
        const int i = (int)(r / C), ch = (int)(r % C);
        double* row = echo_adj + 2 * (size_t)r * (size_t)Ns;
        memset(row, 0, sizeof(double) * 2 * (size_t)Ns);
        double w[64];
        double R[9];
        if (beam) oracle_attitude_matrix(att[3 * i], att[3 * i + 1], att[3 * i + 2], R);
        for (long p = 0; p < npix; ++p) {
            if (beam && !(sensor_sees(R, pix + 3 * p, tx + 3 * i, beam_tan, side) &&
                          sensor_sees(R, pix + 3 * p, rx + 3 * ((size_t)i * C + ch), beam_tan, side)))
                continue;
            oracle_delay d;
            delay_eval(pix + 3 * p, tx + 3 * i, rx + 3 * ((size_t)i * C + ch), vel ? vel + 3 * i : NULL, c, t0,
                       fs, &d);
            oracle_kaiser_sinc_weights(d.f, taps, beta, w, NULL);
            double ph = fc * d.tau;
            ph -= floor(ph);
            const double cs = cos(2.0 * ORACLE_PI * ph), sn = -sin(2.0 * ORACLE_PI * ph);
            const double ir = img[2 * p], ii = img[2 * p + 1];
            const double vr = ir * cs - ii * sn, vi = ir * sn + ii * cs;
            for (int m = 0; m < taps; ++m) {
                const long j = d.j0 + (m - taps / 2 + 1);
                if (j < 0 || j >= Ns) continue;
                row[2 * j] += w[m] * vr;
                row[2 * j + 1] += w[m] * vi;
            }
        }
    }
}

/* Gradient of a real loss L(I) with respect to per-ping position offsets dp_i
 * (the offsets shift the transmitter and every receiver of ping i together),
 * given g(x) = dL/dI*(x) (Wirtinger derivative) at the pixels:
 *   dL/d(dp_i) = 2 Re sum_x sum_c conj(g(x)) dI_ic(x)/d(dp_i),
 *   I_ic(x) = s(u) exp(j 2 pi fc tau),   s(u) = sum_m w_m(f) e[j0 + k_m],
 *   dI_ic/dtau = (fs s'(u) + j 2 pi fc s(u)) exp(j 2 pi fc tau),
 *   s'(u) = sum_m w'_m(f) e[j0 + k_m],
 *   dtau/d(dp_i) = -(u_T + u_R,c) / (c + u_R,c . v_i)  (unit vectors sensor -> pixel;
 *   v_i = 0 for stop-and-hop; with receiver motion u_R is taken at reception).
 * grad: [P][3].  One thread owns one ping.
 * Pinned by: central finite differences of the sharpness through
 * oracle_backproject with offsets applied by oracle_sensor_positions.      */
void oracle_vjp_offsets(int P, int C, const double* tx, const double* rx, double fc, double fs,
                        double c, double t0, int Ns, const double* echo, int taps, double beta,
                        long npix, const double* pix, const double* g, double* grad,
                        const double* att, double beam_tan, int side, const double* vel, int nthreads) {
    set_threads(nthreads);
    const int beam = att != NULL && beam_tan > 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < P; ++i) {
        double gx = 0.0, gy = 0.0, gz = 0.0;
        double w[64], dw[64];
        double R[9];
        if (beam) oracle_attitude_matrix(att[3 * i], att[3 * i + 1], att[3 * i + 2], R);
        for (long p = 0; p < npix; ++p) {
            const double* x = pix + 3 * p;
            if (beam && !sensor_sees(R, x, tx + 3 * i, beam_tan, side)) continue;
            for (int ch = 0; ch < C; ++ch) {
                if (beam && !sensor_sees(R, x, rx + 3 * ((size_t)i * C + ch), beam_tan, side)) continue;
                oracle_delay d;
                delay_eval(x, tx + 3 * i, rx + 3 * ((size_t)i * C + ch), vel ? vel + 3 * i : NULL, c, t0, fs, &d);
                oracle_kaiser_sinc_weights(d.f, taps, beta, w, dw);
                const double* row = echo + 2 * ((size_t)i * C + ch) * (size_t)Ns;
                double sr = 0.0, si = 0.0, dr = 0.0, di = 0.0;
                for (int m = 0; m < taps; ++m) {
                    const long j = d.j0 + (m - taps / 2 + 1);
                    if (j < 0 || j >= Ns) continue;
                    sr += w[m] * row[2 * j];
                    si += w[m] * row[2 * j + 1];
                    dr += dw[m] * row[2 * j];
                    di += dw[m] * row[2 * j + 1];
                }
                double ph = fc * d.tau;
                ph -= floor(ph);
                const double cs = cos(2.0 * ORACLE_PI * ph), sn = sin(2.0 * ORACLE_PI * ph);
                /* a = fs s' + j 2 pi fc s */
                const double ar = fs * dr - 2.0 * ORACLE_PI * fc * si;
                const double ai = fs * di + 2.0 * ORACLE_PI * fc * sr;
                /* dI/dtau = a exp(j phase) */
                const double br = ar * cs - ai * sn, bi = ar * sn + ai * cs;
                /* Re(conj(g) * dI/dtau) */
                const double re = g[2 * p] * br + g[2 * p + 1] * bi;
                const double k = 2.0 * re * (-d.kappa / c);
                gx += k * (d.ut[0] + d.ur[0]);
                gy += k * (d.ut[1] + d.ur[1]);
                gz += k * (d.ut[2] + d.ur[2]);
            }
        }
        grad[3 * i + 0] = gx;
        grad[3 * i + 1] = gy;
        grad[3 * i + 2] = gz;
    }
}

/* Image sharpness S = sum|I|^4 / (sum|I|^2)^2 and its Wirtinger derivative
 *   g = dS/dI* = 2 I (|I|^2 / D^2 - N / D^3),  N = sum|I|^4, D = sum|I|^2.
 * out3 = {S, N, D}; g optional ([n][2]).
 * Pinned by: S = 1 for a single non-zero pixel, S = 1/n for equal
 * magnitudes, scale invariance, and g against central differences.       */
void oracle_sharpness(long n, const double* img, double* out3, double* g) {
    double N = 0.0, D = 0.0;
    for (long p = 0; p < n; ++p) {
        const double a = img[2 * p] * img[2 * p] + img[2 * p + 1] * img[2 * p + 1];
        N += a * a;
        D += a;
    }
    out3[0] = N / (D * D);
    out3[1] = N;
    out3[2] = D;
    if (g) {
        for (long p = 0; p < n; ++p) {
            const double a = img[2 * p] * img[2 * p] + img[2 * p + 1] * img[2 * p + 1];
            const double k = 2.0 * (a / (D * D) - N / (D * D * D));
            g[2 * p] = k * img[2 * p];
            g[2 * p + 1] = k * img[2 * p + 1];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Point-scatterer echo simulator (Eq. 1 with sigma a sum of points, spreading
 * 1/(|x_TX-x||x_RX-x|) omitted), complex baseband after matched filtering:
 *   e[i][c][n] += A_s q_mf(t_n - tau_s) exp(-j 2 pi fc tau_s),  t_n = t0 + n/fs.
 * q_mf is the matched-filter output of a linear FM pulse with rectangular
 * envelope, length T and bandwidth B, normalised to a unit peak:
 *   q_mf(t) = (1 - |t|/T) sinc(B t (1 - |t|/T)),  |t| < T  (0 otherwise);
 * T <= 0 selects the ideal compressed pulse sinc(B t).
 * half_width > 0 limits each point's response to |n - n_tau| <= half_width.
 * scat: [n][5] = (x, y, z, Re A, Im A).  echo is accumulated into.
 * Pinned by: q_mf against a direct numerical correlation of a sampled chirp,
 * unit peak at on-grid delays.  This is an input generator for tests.      */
double oracle_lfm_compressed_pulse(double t, double B, double T) {
    if (T <= 0.0) return sinc_pi(B * t);
    const double a = fabs(t);
    if (a >= T) return 0.0;
    const double r = 1.0 - a / T;
    return r * sinc_pi(B * t * r);
}

void oracle_simulate_points(int P, int C, const double* tx, const double* rx, double fc,
                            double fs, double c, double t0, int Ns, double B, double T,
                            long nscat, const double* scat, int half_width, double* echo,
                            const double* vel, int nthreads) {
    set_threads(nthreads);
    const long rows = (long)P * C;
#pragma omp parallel for schedule(dynamic, 1)
    for (long r = 0; r < rows; ++r) {
        const int i = (int)(r / C), ch = (int)(r % C);
        double* row = echo + 2 * (size_t)r * (size_t)Ns;
        for (long s = 0; s < nscat; ++s) {
            const double* q = scat + 5 * s;
            oracle_delay d;
            delay_eval(q, tx + 3 * i, rx + 3 * ((size_t)i * C + ch), vel ? vel + 3 * i : NULL, c, t0, fs, &d);
            double ph = fc * d.tau;
            ph -= floor(ph);
            const double cs = cos(2.0 * ORACLE_PI * ph), sn = -sin(2.0 * ORACLE_PI * ph);
            const double ar = q[3] * cs - q[4] * sn, ai = q[3] * sn + q[4] * cs;
            long n0 = 0, n1 = Ns - 1;
            if (half_width > 0) {
                const long nc = (long)floor(d.u);
                n0 = nc - half_width;
                n1 = nc + half_width + 1;
                if (n0 < 0) n0 = 0;
                if (n1 > Ns - 1) n1 = Ns - 1;
            }
            for (long n = n0; n <= n1; ++n) {
                const double tn = t0 + (double)n / fs;
                const double a = oracle_lfm_compressed_pulse(tn - d.tau, B, T);
                row[2 * n] += a * ar;
                row[2 * n + 1] += a * ai;
            }
        }
    }
}
