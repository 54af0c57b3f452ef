// Echo simulator: the forward model of Eq. 1 for point scatterers (spreading
// loss omitted), complex baseband after matched filtering:
//   e[i][c][k] += A q(t_k - tau) exp(-j 2 pi fc tau),  t_k = t0 + k / fs,
//   tau = (|x_s - x_TX,i| + |x_s - x_RX,i,c|) / c,
//   q(t) = (1 - |t|/T) sinc(B t (1 - |t|/T)),  |t| < T,
// the autocorrelation of a linear FM pulse of length T and bandwidth B with a
// rectangular envelope, normalised to a unit peak (T <= 0 selects sinc(B t)).
// With a receiver velocity set, tau solves c tau = |x_s - x_TX| + |x_s - x_RX - v tau|.
// With the seabed refraction model, a leg from a sensor above the interface to
// a scatterer below it counts |P - s| + n |x_s - P| water metres, P the
// crossing where the travel time is stationary (Snell's law, solved by
// bisection in FP64).
// One block per (ping, channel) row; FP64 delay and carrier phase per
// (row, scatterer); FP32 pulse samples accumulated with global atomics.
#include "sas_common.cuh"

namespace sas {
namespace {

// Length in water metres of the leg from sensor s to point x: straight, or
// with the refraction model (n > 0) and s above / x below the interface
// z = z_int, |W| + n |V| with the crossing at horizontal run xi from the
// sensor where xi / |W| = n (rho - xi) / |V| (the left side minus the right
// increases with xi; bisection on [0, rho] until the bracket is below 1e-12 of
// the run: the length is stationary at the crossing, so its error is of the
// bracket's square).
__device__ double leg_length(const double* sv, double x, double y, double z, double z_int, double n) {
    const double hx = x - sv[0], hy = y - sv[1], hz = z - sv[2];
    if (!(n > 0.0) || !(sv[2] < z_int) || !(z > z_int)) return sqrt(hx * hx + hy * hy + hz * hz);
    const double a = z_int - sv[2], b = z - z_int, rho = sqrt(hx * hx + hy * hy);
    double lo = 0.0, hi = rho;
    for (int it = 0; it < 200 && hi - lo > 1e-12 * (rho + 1.0); ++it) {
        const double m = 0.5 * (lo + hi), sg = rho - m;
        if (m * sqrt(sg * sg + b * b) > n * sg * sqrt(m * m + a * a))
            hi = m;
        else
            lo = m;
    }
    const double xi = 0.5 * (lo + hi), sg = rho - xi;
    return sqrt(xi * xi + a * a) + n * sqrt(sg * sg + b * b);
}

__global__ void simulate_points_kernel(const double* __restrict__ tx, const double* __restrict__ rx,
                                       const double* __restrict__ vel, int C, int Ns, double t0, double fs,
                                       double fc, double inv_c, const double* __restrict__ scat, long long nscat,
                                       float B, float T, int half_width, double z_int, double n_refr,
                                       float2* __restrict__ echo) {
    const long long row = blockIdx.x;
    const int i = (int)(row / C);
    const double* t = tx + 3 * (size_t)i;
    const double* r = rx + 3 * (size_t)row;
    float2* e = echo + (size_t)row * Ns;
    const float inv_fs = (float)(1.0 / fs);
    for (long long s = 0; s < nscat; ++s) {
        const double* q = scat + 5 * s;
        const double bx = q[0] - r[0], by = q[1] - r[1], bz = q[2] - r[2];
        const double rt = leg_length(t, q[0], q[1], q[2], z_int, n_refr);
        double tau = (rt + leg_length(r, q[0], q[1], q[2], z_int, n_refr)) * inv_c;
        if (vel) {
            // receiver moving during reception: c tau = |x - x_TX| + |x - x_RX - v tau|
            const double* v = vel + 3 * (size_t)i;
            for (int it = 0; it < 12; ++it) {
                const double wx = bx - v[0] * tau, wy = by - v[1] * tau, wz = bz - v[2] * tau;
                const double t2 = (rt + sqrt(wx * wx + wy * wy + wz * wz)) * inv_c;
                const double step = fabs(t2 - tau);
                tau = t2;
                if (step <= 1e-16 * tau) break;
            }
        }
        const double u = (tau - t0) * fs;
        double ph = fc * tau;
        ph -= floor(ph);
        double sn, cs;
        sincospi(-2.0 * ph, &sn, &cs);
        const float Ar = (float)(q[3] * cs - q[4] * sn), Ai = (float)(q[3] * sn + q[4] * cs);
        const long long kc = (long long)floor(u);
        long long k0 = 0, k1 = Ns - 1;
        if (half_width > 0) {
            k0 = max(0LL, kc - half_width);
            k1 = min((long long)Ns - 1, kc + half_width + 1);
        }
        const float frac = (float)(u - (double)kc);
        for (long long k = k0 + threadIdx.x; k <= k1; k += blockDim.x) {
            const float dt = ((float)(k - kc) - frac) * inv_fs;   // t_k - tau
            float a;
            if (T <= 0.f) {
                const float x = B * dt;
                a = (x == 0.f) ? 1.f : sinpif(x) / (3.14159265358979f * x);
            } else {
                const float ad = fabsf(dt);
                if (ad >= T) continue;
                const float rr = 1.f - ad / T;
                const float x = B * dt * rr;
                a = rr * ((x == 0.f) ? 1.f : sinpif(x) / (3.14159265358979f * x));
            }
            atomicAdd(e + k, make_float2(a * Ar, a * Ai));
        }
    }
}

}  // namespace
}  // namespace sas

using namespace sas;

extern "C" int sas_simulate_points(sas_geometry_t h, const double* d_scat, int64_t n, double bandwidth, double pulse_T,
                                   int32_t half_width, void* d_echo, void* stream) {
    if (!h || !d_echo || n < 0 || (n > 0 && !d_scat) || !(bandwidth > 0) || half_width < 0) {
        set_error("sas_simulate_points: bad argument");
        return SAS_ERR_ARG;
    }
    if (h->c_sed > 0.0 && h->has_vel) {
        set_error("sas_simulate_points: the refraction model does not combine with receiver motion");
        return SAS_ERR_UNSUPPORTED;
    }
    if (n == 0) return SAS_OK;
    const unsigned rows = (unsigned)((long long)h->P * h->C);
    simulate_points_kernel<<<rows, 256, 0, (cudaStream_t)stream>>>(
        h->d_tx, h->d_rx, h->has_vel ? h->d_vel : nullptr, h->C, h->Ns, h->sig.t0, h->sig.fs, h->sig.fc, 1.0 / h->sig.c, d_scat, n, (float)bandwidth,
        (float)pulse_T, half_width, h->z_int, h->c_sed > 0.0 ? h->sig.c / h->c_sed : 0.0, (float2*)d_echo);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}
