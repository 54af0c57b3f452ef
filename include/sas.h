/*
 * sas.h -- C ABI of the GB300 time-domain backprojection library (libsas).
 *
 * The library forms synthetic-aperture-sonar images by time-domain
 * backprojection (TDBP): for every pixel or voxel x, every ping i and every
 * receiver channel c it evaluates the two-way delay
 *     tau_ic(x) = (|x - x_TX,i| + |x - x_RX,i,c|) / c_sound,
 * interpolates the range-compressed complex baseband echo at that delay and
 * accumulates it rotated by exp(+j 2 pi f_c tau) into the image:
 *     I(x) = sum_i sum_c s_ic(u_ic(x)) exp(+j 2 pi f_c tau_ic(x)),
 *     u = (tau - t0) f_s,   s(u) = sum_{k=-3..4} w_k(frac u) e[i][c][floor u + k].
 * This is the per-pixel inversion of the forward model, Eq. 1 of arXiv
 * 2101.05888 (ASASIN), Sec. II-A; samples outside [0, Ns) read as zero.
 * Transmitter/receiver positions follow Eq. 2 (attitude) and the lever arms of
 * Sec. II-C, in the north-east-down frame of Sec. II-B.
 *
 * Conventions for every call:
 *  - Return value: SAS_OK (0) or a negative sas_status; no exception crosses
 *    the ABI.  sas_last_error() gives a message for the calling thread.
 *  - Calls are asynchronous and stream-ordered on the CUDA stream passed in
 *    (NULL = legacy default stream).  Device faults detected inside kernels
 *    (a bounded wait that ran out) are recorded in a per-handle status word and
 *    reported by sas_sync_status().
 *  - "Host" pointers are read during the call (the caller may free them when
 *    the call returns).  "Device" pointers are caller-owned GPU memory that
 *    must stay valid until the stream work completes.
 *  - A handle may be used from one stream at a time.
 *  - Complex arrays are interleaved (re, im) float32 pairs (complex64).
 *  - Arrays are C-contiguous in the order written, last index fastest.
 */
#ifndef SAS_H
#define SAS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAS_VERSION 10000 /* 1.0.0 */

typedef enum {
    SAS_OK = 0,
    SAS_ERR_ARG = -1,         /* invalid argument (null pointer, bad size, ...) */
    SAS_ERR_CUDA = -2,        /* a CUDA runtime/driver call failed */
    SAS_ERR_OOM = -3,         /* device allocation failed */
    SAS_ERR_TIMEOUT = -4,     /* a kernel's bounded wait ran out (results invalid) */
    SAS_ERR_UNSUPPORTED = -5, /* valid but unsupported configuration */
    SAS_ERR_STATE = -6,       /* call out of order (e.g. no echo uploaded) */
    SAS_ERR_CHECK = -7        /* checked build: a kernel's index check fired (results invalid) */
} sas_status;

/* Storage type of the echo inside the handle. */
typedef enum {
    SAS_ECHO_C64 = 0,      /* complex64: float32 (re, im) */
    SAS_ECHO_C32_F16 = 1,  /* complex as two float16, with a float32 scale per (ping, channel) */
    SAS_ECHO_C32_BF16 = 2  /* complex as two bfloat16, with a float32 scale per (ping, channel) */
} sas_echo_dtype;

/* Signal description (Eq. 1): carrier fc [Hz], complex baseband sample rate
 * fs [Hz], sound speed c [m/s], t0 = delay of echo sample 0 after transmit
 * [s], n_samples = samples per (ping, channel) row.  n_samples must be a
 * multiple of 4 (16-byte rows for the bulk-copy engine). */
typedef struct {
    double fc, fs, c, t0;
    int32_t n_samples;
} sas_signal;

/* Navigation (Sec. II-B/C).  All arrays host, FP64, NED metres / radians.
 *   ping_pos [P][3]  vehicle reference point per ping
 *   ping_att [P][3]  (roll, pitch, yaw) per ping, rotation of Eq. 2
 *   tx_lever [3]     transmitter lever arm, body frame
 *   rx_lever [C][3]  receiver lever arms, body frame
 * Stop-and-hop: transmitter and receivers sit at their ping-time positions. */
typedef struct {
    int32_t n_pings, n_rx;
    const double* ping_pos;
    const double* ping_att;
    const double* tx_lever;
    const double* rx_lever;
} sas_nav;

/* Pixel grid: pixel (ix, iy, iz) sits at (x0 + ix dx, y0 + iy dy, z0 + iz dz);
 * images are [nz][ny][nx] complex64 with ix fastest.  2D images use nz = 1
 * (dz ignored). */
typedef struct {
    double x0, y0, z0, dx, dy, dz;
    int32_t nx, ny, nz;
} sas_grid;

typedef enum {
    SAS_INTERP_KAISER_SINC = 0, /* normalised Kaiser-windowed sinc, `taps` taps, shape kaiser_beta */
    SAS_INTERP_TABLE = 1        /* user taps tabulated on a uniform fraction grid (see below) */
} sas_interp_kind;

/* Fractional-delay interpolator.  The paper does not name its interpolator;
 * the library's default is the Kaiser-windowed sinc normalised to unit sum:
 *   w_k(f) = v(f - k) / sum_k' v(f - k'),
 *   v(d)   = sinc(d) I0(beta sqrt(1 - (2d/taps)^2)) / I0(beta), |d| < taps/2,
 * taps k = -taps/2+1 .. taps/2 around floor(u), f = u - floor(u).
 * SAS_INTERP_TABLE: d_table is a device FP32 array [table_n + 1][taps] of tap
 * values at f = j / table_n (j = 0 .. table_n), e.g. a tabulated learned
 * interpolator; values between rows are linear in f.
 * Only taps = 8 is supported by the backprojection kernels. */
typedef struct {
    int32_t kind;
    int32_t taps;
    double kaiser_beta;
    int32_t table_n;
    const float* d_table;
} sas_interp;

typedef struct sas_geometry_s* sas_geometry_t;

/* Library version (SAS_VERSION) and the message of the last failed call on
 * this thread ("" if none).  The string stays valid until the next call. */
int sas_version(void);
const char* sas_last_error(void);

/* Creates a handle on the current CUDA device: copies the navigation and
 * signal description, allocates the handle's device slab and computes the
 * transmitter and receiver positions per ping (Eq. 2 rotation of the lever
 * arms plus the vehicle position; per-ping offsets start at zero) with an FP64
 * kernel on `cuda_stream`.  *out receives the handle.
 * Errors: SAS_ERR_ARG (null pointers, P or C < 1, n_samples < 8 or not a
 * multiple of 4, non-positive fs or c), SAS_ERR_OOM, SAS_ERR_CUDA. */
int sas_geometry_create(const sas_nav* nav, const sas_signal* sig, void* cuda_stream,
                        sas_geometry_t* out);

/* Sets per-ping position offsets dp [P][3] (FP64, metres, added to the vehicle
 * position, hence to the transmitter and every receiver of that ping) and
 * recomputes the sensor positions.  offsets == NULL resets them to zero.
 * on_device: 0 = host array, 1 = device array.  This is the variable that
 * sas_backproject_adjoint differentiates against (autofocus). */
int sas_geometry_set_offsets(sas_geometry_t h, const double* offsets, int on_device,
                             void* cuda_stream);

/* Beam field of view (Sec. II-C: pixels outside the transmit or receive beam
 * are not integrated).  Every transducer gets an azimuth beam of full width
 * beam_width [rad] centred on the vehicle's side axis (side = +1: body +y,
 * starboard; -1: port); elevation is unrestricted.  Sensor s of ping i sees
 * pixel x iff b = R_i^T (x - x_s) has side b_y > 0 and
 * |b_x| <= tan(beam_width/2) side b_y; a (ping, channel) term is integrated
 * iff the transmitter and that receiver both see x.  Applies to every later
 * backprojection and adjoint call; beam_width <= 0 switches it off (the
 * default).  The kernels skip (ping, channel, tile) blocks that a
 * conservative test of the tile corners proves invisible (ray culling) and
 * test pixels individually only in tiles on a beam edge, so the result equals
 * the per-pixel definition.  Errors: SAS_ERR_ARG (beam_width >= pi, bad side). */
int sas_geometry_set_beam(sas_geometry_t h, double beam_width, int side);

/* Receiver motion during reception (Sec. II-D: transmission is
 * instantaneous and the platform keeps moving while the echo comes in; the
 * stop-and-hop approximation drops that motion).  vel [P][3] (FP64, m/s,
 * NED): the velocity of ping i's receivers during its reception; host
 * (on_device = 0, read before the call returns) or device (on_device = 1,
 * copied on the stream).  With a velocity the two-way delay of pixel x solves
 * c tau = |x - x_TX,i| + |x - x_RX,i,c - v_i tau| (transmitter fixed at the
 * ping time); every later backprojection, adjoint, offset gradient and
 * simulation uses it.  vel == NULL returns to stop-and-hop (the default).
 * Beam tests keep the ping-time sensor positions.  Errors: SAS_ERR_ARG,
 * SAS_ERR_CUDA. */
int sas_geometry_set_velocity(sas_geometry_t h, const double* vel, int on_device, void* cuda_stream);

/* Refraction at the seabed (Sec. III-B: imaging below the seafloor needs a
 * refraction model in the propagation time).  A flat interface z = z_interface
 * (NED, metres) with water above (the signal's sound speed c) and sediment
 * below (sound speed c_sediment, m/s).  A leg from a sensor above the
 * interface to a pixel strictly below it (z > z_interface) crosses the
 * interface where its travel time is stationary (Fermat; Snell's law) and
 * counts L = |P - s| + (c / c_sediment) |x - P| water metres; every other leg
 * is straight.  Applies to the forward backprojection (2D and 3D), the linear
 * adjoint and the offset gradient (the derivative of a refracted leg's length
 * with respect to its sensor is minus the unit vector towards the crossing
 * point) and the echo simulator of every later call; c_sediment <= 0
 * switches the model off (the default).  Those calls return
 * SAS_ERR_UNSUPPORTED when the handle also has a velocity
 * (sas_geometry_set_velocity) or, except the simulator, a beam
 * (sas_geometry_set_beam).
 * Errors: SAS_ERR_ARG (null handle, non-finite arguments). */
int sas_geometry_set_refraction(sas_geometry_t h, double z_interface, double c_sediment);

/* Copies the current sensor positions to device arrays d_tx [P][3] and
 * d_rx [P][C][3] (FP64).  Either may be NULL. */
int sas_geometry_positions(sas_geometry_t h, double* d_tx, double* d_rx, void* cuda_stream);

/* Releases the handle and all device memory it owns (synchronises the device). */
int sas_geometry_destroy(sas_geometry_t h);

/* Stores the echo in the handle.  echo: complex64 [P][C][Ns], host
 * (on_device = 0) or device (on_device = 1).  store_dtype selects the storage:
 * SAS_ECHO_C64 copies as is; the 16-bit types divide each (ping, channel) row
 * by its largest |component| (kept as a float32 scale and re-applied inside
 * the kernels) and round to float16 / bfloat16 on the device.  Replaces any
 * previous echo.  Errors: SAS_ERR_ARG, SAS_ERR_OOM, SAS_ERR_CUDA. */
int sas_echo_upload(sas_geometry_t h, const void* echo, int on_device, int store_dtype,
                    void* cuda_stream);

/* Copies the stored echo, converted back to complex64 (scale applied), into
 * d_out [P][C][Ns] (device).  For inspecting the quantised echo. */
int sas_echo_download(sas_geometry_t h, void* d_out, void* cuda_stream);

/* 2D backprojection onto the grid plane z = z0 (grid->nz must be 1).
 * d_image: complex64 [ny][nx], device.  accumulate = 0 overwrites the image,
 * 1 adds to it (e.g. to stream pings through several echo uploads).
 * Errors: SAS_ERR_ARG, SAS_ERR_STATE (no echo), SAS_ERR_UNSUPPORTED (taps != 8,
 * a tile's delay span too long for the staging buffers), SAS_ERR_CUDA. */
int sas_backproject_2d(sas_geometry_t h, const sas_grid* grid, const sas_interp* interp,
                       void* d_image, int accumulate, void* cuda_stream);

/* 3D backprojection, voxel grid [nz][ny][nx] (Sec. III-B layered volume).
 * Same contract as sas_backproject_2d. */
int sas_backproject_3d(sas_geometry_t h, const sas_grid* grid, const sas_interp* interp,
                       void* d_image, int accumulate, void* cuda_stream);

/* Adjoints of the backprojection B (echo -> image) on `grid` (2D or 3D):
 *  - d_echo_adj != NULL: linear adjoint  e_adj = B^H d_grad_image, complex64
 *    [P][C][Ns] device, overwritten:
 *        e_adj[i][c][floor u + k] += w_k(frac u) exp(-j 2 pi fc tau) I(x);
 *  - d_grad_offsets != NULL: gradient of a real loss L with respect to the
 *    per-ping offsets, [P][3] FP64 device, overwritten, given
 *    d_grad_image = dL/dI* (complex64 image):
 *        dL/d(dp_i) = 2 Re sum_x sum_c conj(g(x)) dI_ic(x)/d(dp_i).
 *    Image tiles are recomputed (not stored); per-tile partial sums are
 *    reduced in a fixed order (deterministic).
 * At least one output must be non-NULL. */
int sas_backproject_adjoint(sas_geometry_t h, const sas_grid* grid, const sas_interp* interp,
                            const void* d_grad_image, void* d_echo_adj, double* d_grad_offsets,
                            void* cuda_stream);

/* Image sharpness S = sum|I|^4 / (sum|I|^2)^2 over n complex64 values
 * (d_image, device).  d_out3 (device, FP64 [3]) receives {S, N = sum|I|^4,
 * D = sum|I|^2}; if d_grad != NULL it receives g = dS/dI* =
 * 2 I (|I|^2/D^2 - N/D^3) (complex64 [n], device).  Sums are FP64 and
 * deterministic.  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_sharpness(const void* d_image, int64_t n, double* d_out3, void* d_grad, void* cuda_stream);

/* sas_sharpness for callers that may not allocate device memory while they
 * run (for example a vehicle-borne processor that reserves all of its GPU
 * memory at start-up, or a host framework whose memory manager forbids
 * cudaMalloc/cudaFree because they synchronise the device).  The paper has no
 * counterpart; this is a service entry point of the library.
 * Same arguments and outputs as sas_sharpness; the sums agree with it to FP64
 * rounding (a different block split).  It allocates nothing: its per-block
 * partial sums live in a 64 KiB array compiled into the library, which every
 * GPU that loads the library holds until the process exits.
 * Limits and rules:
 *  - n <= 67,108,864 (16384 elements per block x 4096 blocks); larger n is
 *    rejected with SAS_ERR_ARG before anything is launched.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents;
 *    each call writes every slot it later reads, so nothing needs clearing.
 *    Calls whose GPU work overlaps (different streams, no ordering) race on
 *    the array and give wrong results: order them. */
int sas_sharpness_static(const void* d_image, int64_t n, double* d_out3, void* d_grad, void* cuda_stream);

/* Evaluates the interpolator's taps at n fractions f (device FP32 [n]) into
 * d_taps (device FP32 [n][taps]) exactly as the backprojection kernels apply
 * them, and writes to *d_max_err (device FP64, may be NULL) the largest
 * deviation of that form from the interpolator's definition over a fine
 * fraction grid.  The kernels apply each tap's weight as a polynomial in the
 * fraction on each half of the sample interval (a Farrow form, Sec. II-A's
 * interpolation evaluated without a per-update tap table): a cubic for
 * complex64 echoes, in the gradient pass and in the adjoint, and a quadratic
 * for 16-bit echoes in the forward pass.  sas_interp_eval evaluates the cubic
 * form; sas_interp_eval_form the one of the given degree (3 or 2; any other
 * value is SAS_ERR_ARG). */
int sas_interp_eval(const sas_interp* interp, const float* d_f, int64_t n, float* d_taps,
                    double* d_max_err, void* cuda_stream);
int sas_interp_eval_form(const sas_interp* interp, int degree, const float* d_f, int64_t n, float* d_taps,
                         double* d_max_err, void* cuda_stream);

/* Echo simulator (Eq. 1 for point scatterers, spreading loss omitted),
 * complex baseband after matched filtering, using the handle's current sensor
 * positions.  Adds to d_echo (device complex64 [P][C][Ns]):
 *   e[i][c][k] += A q(t_k - tau) exp(-j 2 pi fc tau),  t_k = t0 + k/fs,
 *   q(t) = (1 - |t|/T) sinc(B t (1 - |t|/T)) for |t| < T, else 0
 * (matched-filter output of a linear FM pulse of length T = pulse_T and
 * bandwidth B = bandwidth with a rectangular envelope, unit peak;
 * pulse_T <= 0 gives sinc(B t)).  d_scat: device FP64 [n][5] =
 * (x, y, z, Re A, Im A).  half_width > 0 limits each response to samples
 * |k - (tau - t0) fs| <= half_width (0 = whole row). */
int sas_simulate_points(sas_geometry_t h, const double* d_scat, int64_t n, double bandwidth, double pulse_T,
                        int32_t half_width, void* d_echo, void* cuda_stream);

/* ---- Learned interpolator (MLP 1 -> 64 -> 64 -> 8, GELU, FP16 weights) ----
 * Parameters are a flat FP32 master vector theta [SAS_MLP_NPARAMS] in the
 * order W1 [64][1], b1 [64], W2 [64][64] ([out][in]), b2 [64], W3 [8][64],
 * b3 [8]; the network input is x = 2 f - 1.  Kernels round the weights to
 * FP16 and compute in FP32:  a1 = gelu(W1 x + b1), a2 = gelu(W2 a1 + b2),
 * t = W3 a2 + b3,  gelu(z) = z/2 (1 + erf(z/sqrt 2)).
 * The interpolator's taps are the taps of a fixed prior, the normalised
 * 8-tap Kaiser-sinc at beta = prior_beta (the plain interpolator), plus the
 * network's correction t; prior_beta < 0 means no prior (taps = t).  The
 * network is trained on residual targets (the 32-tap interpolation minus the
 * prior's), so the loss below is the error of prior + network. */
#define SAS_MLP_NPARAMS 4808

/* Training windows from an echo (device complex64 [rows][Ns]): for n draws
 * (d_frac [n] FP32 fractions, d_row [n] int32 rows, d_pos [n] int32 sample
 * indices) writes the 8-sample window e[row][pos-3 .. pos+4] to d_windows
 * (complex64 [n][8]) and to d_targets (complex64 [n]) the 32-tap Kaiser-sinc
 * (beta = target_beta) interpolation at pos + frac, minus the prior's 8-tap
 * interpolation of the window if prior_beta >= 0 (both sums in FP64).
 * Samples outside the row read as zero. */
int sas_mlp_make_windows(const void* d_echo, int32_t rows, int32_t n_samples, const float* d_frac,
                         const int32_t* d_row, const int32_t* d_pos, int64_t n, double target_beta,
                         double prior_beta, void* d_windows, void* d_targets, void* cuda_stream);

/* Loss L = mean_b |sum_m t_m(f_b) s_b,m - y_b|^2 and its gradient w.r.t. theta
 * (device FP32 [SAS_MLP_NPARAMS], overwritten) on a batch of n windows.
 * d_loss: device FP32 [1].  d_work: device scratch of sas_mlp_workspace_bytes(n). */
int64_t sas_mlp_workspace_bytes(int64_t n);
int sas_mlp_loss_grad(const float* d_theta, const float* d_frac, const void* d_windows,
                      const void* d_targets, int64_t n, float* d_loss, float* d_grad, void* d_work,
                      void* cuda_stream);

/* One Adam update (Kingma & Ba) of theta with moments m, v (all device FP32
 * [SAS_MLP_NPARAMS]); step counts from 1. */
int sas_mlp_adam(float* d_theta, const float* d_grad, float* d_m, float* d_v, int32_t step,
                 float lr, float beta1, float beta2, float eps, void* cuda_stream);

/* Tabulates the interpolator's taps (the prior's, FP64, when prior_beta >= 0,
 * plus the network's) at f = j / table_n, j = 0 .. table_n, into d_table_out
 * (device FP32 [table_n + 1][8]) for use as SAS_INTERP_TABLE. */
int sas_interp_tabulate_mlp(const float* d_theta, int32_t table_n, double prior_beta, float* d_table_out,
                            void* cuda_stream);

/* Waits for the stream, then reports and clears the handle's device status:
 * SAS_ERR_TIMEOUT if a kernel's bounded wait ran out since the last check,
 * else SAS_ERR_CHECK if (checked build only) a backprojection or adjoint
 * kernel computed a Farrow-row index outside the window the host sized for
 * its tile (the kernel clamped it: no access left the buffer, but the
 * result is wrong).
 * After a timeout the results of the calls since the last check are invalid,
 * and a kernel may have left while one of its own bulk copies was still in
 * flight: treat the device state as suspect and recreate the handle (and
 * re-upload the echo) before relying on further results. */
int sas_sync_status(sas_geometry_t h, void* cuda_stream);

/* Build options of the loaded library: bit 0 set when it was compiled with
 * SAS_CHECKED (the checked build: index checks in the kernels record what
 * they find in the status word instead of only clamping; slower). */
int sas_build_flags(void);

/* ---- Data conditioning (Sec. II-E) and range compression ----------------
 * Rows are complex64 [rows][n], device, caller-owned; d_out may equal d_in.
 * Calls are stream-ordered and allocate their scratch on the stream. */

/* Range compression of raw echo rows by the transmitted replica p [L]
 * (complex64, device): y[k] = sum_l e[k + l] conj(p[l]) / sum_l |p[l]|^2
 * for k < n, samples past the row reading zero (an echo of A p(t - tau)
 * peaks at the sample of tau with value A).  FP32 FFT overlap-save.
 * 1 <= L <= 4096.  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_matched_filter(const void* d_raw, int64_t rows, int32_t n, const void* d_replica, int32_t L, void* d_out,
                       void* cuda_stream);

/* Spectral whitening, Eq. 9: P(f) = mean over the rows of |FFT(e)(f)|^2,
 * G(f) = 1 / (gamma mean_f P + P(f)) scaled so that max G = 1 (the smallest
 * attenuation is 0 dB), applied as a power gain: rows = IFFT(FFT(e) sqrt G).
 * n a power of two in [4, 16384]; gamma >= 0.  d_gain: optional device
 * float [n] receiving sqrt G.  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_whiten(const void* d_in, void* d_out, int64_t rows, int32_t n, double gamma, float* d_gain,
               void* cuda_stream);

/* Time-varying gain, Eq. 10: P(t) = median over the rows of the FP32 power
 * |e(t)|^2 (re*re + im*im rounded to FP32; an even count takes the mean of
 * the two middle values), G(t) = 1 / (alpha mean_t P + P(t)), applied as a
 * power gain: rows times sqrt G(t) (no correction where alpha = 0 and the
 * median is 0).  Optional outputs: d_gain float [n]
 * (sqrt G), d_median double [n] (P).  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_tvg(const void* d_in, void* d_out, int64_t rows, int32_t n, double alpha, float* d_gain, double* d_median,
            void* cuda_stream);

/* Dynamic range compression, Eqs. 11-12: I_n = |I| / max |I| (FP32, |I| the
 * correctly rounded magnitude), q = (b - b m) / (m - b m) with m the median
 * of I_n (even count: mean of the two middle values), and
 * d_out[i] = q I_n / ((q - 1) I_n + 1) (float, [0, 1], the median pixel
 * maps to b; a median of 1 gives the identity map, a median of 0 sends every
 * non-zero pixel to 1).  d_image complex64 [npix]; 0 < b < 1.  d_stats: optional
 * device double [3] = {q, m, max |I|}.  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_drc(const void* d_image, int64_t npix, double b, float* d_out, double* d_stats, void* cuda_stream);

/* Ray-culling counts (Sec. II-C: blocks of pixels outside the beams are
 * pruned before the per-pixel test) accumulated by the forward and
 * offset-gradient backprojections of this handle since the last reset:
 * out[0] = candidate (ping, channel, image tile) blocks, out[1] = blocks
 * computed (not culled), out[2] = computed blocks on a beam edge, whose pixels
 * are tested one by one.  With no beam all candidates are computed and none
 * is on an edge.  Waits for the stream; reset != 0 zeroes the counts after
 * reading.  out: host array of 3.  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_cull_stats(sas_geometry_t h, long long* out, int reset, void* cuda_stream);

/* Test hook for failure detection: when skip != 0 the next backprojection
 * launches do not issue their bulk copies and use a wait limit of
 * wait_limit_ms, so their waits run out and the kernels return early with the
 * timeout status set (no fault, no trap).  skip = 0 restores normal operation. */
int sas_debug_starve_copies(sas_geometry_t h, int skip, int32_t wait_limit_ms);

/* ---- Displaced-phase-centre (DPC) micronavigation (Sec. II-D, Eqs. 3-8) ----
 *
 * Kinematics: ping i leaves at T_i from the platform position p_i; while its
 * echo comes in the platform moves with the constant velocity v_i (p = v t,
 * transmission instantaneous), and p_{i+1} = p_i + v_i dt_i.  Transmitter:
 * p_i + R_i l_TX; receiver c at time t after transmission: p_i + v_i t +
 * R_i l_c (R_i of Eq. 2, attitude constant during the reception).  DPC pairs:
 * receiver c + shift of ping i with receiver c of ping i + 1 (c = 0 .. C - 1 -
 * shift): their phase centres overlap when the array advances shift half
 * element pitches per ping.
 *
 * Measurement layout ("DPC layout"): index m = (i (C - shift) + c) K + k for
 * ping pair i = 0 .. P - 2, receiver c = 0 .. C - shift - 1, window
 * k = 0 .. K - 1; M = (P - 1)(C - shift) K. */

/* Time-delay estimation between the DPC pairs of the echo stored in h (after
 * the method the paper cites: coarse delay from the magnitude of the complex
 * correlation, fine delay from its phase).  For every measurement:
 * R(tau) = sum_n e[i+1][c][n] conj(e[i][c+shift][n - tau]) over the W samples
 * n in [centre_k - W/2, centre_k - W/2 + W) and lags |tau| <= max_lag (samples
 * outside a row read zero).  coarse = (lag of max |R|, refined by the
 * parabola through |R| at the peak and its two neighbours; no refinement at
 * the edge lags) / fs  [s]; fine = -arg R(coarse) / (2 pi fc) [s, in
 * (-1/(2 fc), 1/(2 fc)]], R(coarse) by the same three-point interpolation of
 * the complex values; rho = |R(peak lag)| / sqrt(sum |e2|^2 sum |e1 shifted|^2).
 * The unwrapped delay is fine + k / fc for the integer k nearest to a
 * reference (sas_dpc_model_delays of a coarse solution).  d_centres: [K]
 * int32 device (sample indices); outputs: FP64 device arrays [M] in the DPC
 * layout, any may be NULL.  FP32 correlation sums.  Constraints: 1 <= W <=
 * 4096, 0 <= max_lag <= 15, 0 <= shift < C, P >= 2.  Errors: SAS_ERR_ARG,
 * SAS_ERR_STATE (no echo), SAS_ERR_CUDA. */
int sas_dpc_delays(sas_geometry_t h, int32_t shift, const int32_t* d_centres, int32_t K, int32_t W,
                   int32_t max_lag, double* d_coarse, double* d_fine, double* d_rho, void* cuda_stream);

/* The motion problem of Eq. 8 (all arrays FP64 on the device, caller-owned). */
typedef struct sas_dpc_problem {
    int32_t P, C, shift, K;     /* pings, receivers per ping, DPC shift, windows per ping pair */
    int32_t side;               /* imaging side: +1 starboard (body +y), -1 port */
    double c;                   /* sound speed [m/s] */
    double lambda1, lambda2;    /* Eq. 8 weights of Eq. 6 (smoothness) and Eq. 7 (DVL) */
    double huber;               /* > 0: Eq. 3 on r / huber, r = c g [m]; <= 0: squares (Eq. 5) */
    const double* d_p0;         /* [3] platform position at ping 0 (NED) */
    const double* d_vx;         /* [P] surge velocity (known) */
    const double* d_att;        /* [P][3] roll, pitch, yaw */
    const double* d_dt;         /* [P-1] ping intervals */
    const double* d_tx_lever;   /* [3] */
    const double* d_rx_lever;   /* [C][3] */
    const double* d_t;          /* [K] window centre times [s after transmission] */
    const double* d_delay;      /* [M] measured delays [s] (DPC layout) */
    const double* d_weight;     /* [M] weights (e.g. rho) or NULL for 1 */
    const double* d_z_dvl;      /* [P] platform depth from the DVL (Eq. 7) */
    const double* d_ps;         /* [M][3] footprints (sas_dpc_footprints) */
} sas_dpc_problem;

/* Footprints p_s of Eq. 4: for measurement (i, c, k) the point of the flat
 * seafloor z = 0 abeam of ping i's phase centre (midpoint of its transmitter
 * and receiver c + shift) on the imaging side, at slant range c t_k / 2 from
 * it, with the positions integrated from the velocities (d_vy, d_vz) [P]
 * (the navigation prior).  d_ps: [M][3].  pr->d_ps, d_delay, d_weight and
 * d_z_dvl are not read.  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_dpc_footprints(const sas_dpc_problem* pr, const double* d_vy, const double* d_vz, double* d_ps,
                       void* cuda_stream);

/* The delays that make Eq. 4 vanish for the velocities (d_vy, d_vz):
 * (path of ping i+1 - path of ping i) / c, with both receivers at t_k; [M]
 * FP64.  d_delay and d_weight are not read.  Errors: SAS_ERR_ARG, SAS_ERR_CUDA. */
int sas_dpc_model_delays(const sas_dpc_problem* pr, const double* d_vy, const double* d_vz, double* d_out,
                         void* cuda_stream);

/* Minimises Eq. 8 = sum_m w_m h(r_m) + lambda1 (Eq. 6) + lambda2 (Eq. 7) over the
 * sway and heave velocities (d_vy, d_vz) [P] (in: start, out: solution) by
 * Levenberg-Marquardt in FP64 (Gauss-Newton normal equations with
 * Marquardt's diagonal damping; Huber by iteratively reweighted residuals).
 * Eq. 6: v''[i] = v[i+1] - 2 v[i] + v[i-1]; Eq. 7: (p_z,i - z_dvl[i]) with
 * p_z,i = p_z,0 + sum_{n<i} v_z[n] dt_n.  The normal equations are solved in
 * the equivalent variables (positions p_1 .. p_{P-1} and the last velocity),
 * where they are banded (half-bandwidth 7).  At most max_iter accepted steps;
 * stops when the loss or the step stalls (relative 1e-14).  h_loss (host,
 * may be NULL): the final Eq. 8 value; h_iters (host, may be NULL): accepted
 * steps.  Synchronises the stream.  Errors: SAS_ERR_ARG, SAS_ERR_OOM,
 * SAS_ERR_CUDA. */
int sas_dpc_solve(const sas_dpc_problem* pr, double* d_vy, double* d_vz, int32_t max_iter, double* h_loss,
                  int32_t* h_iters, void* cuda_stream);

/* Test hook: the banded solve inside sas_dpc_solve streams its rows through
 * shared memory in chunks of 512 rows; rows (a power of two in [8, 512]) sets
 * a smaller chunk for the following calls of this process, so that small
 * problems cross chunk boundaries; rows = 0 restores 512.  The result does
 * not depend on it.  Errors: SAS_ERR_ARG. */
int sas_debug_dpc_solve_chunk(int32_t rows);

#ifdef __cplusplus
}
#endif

#endif /* SAS_H */
