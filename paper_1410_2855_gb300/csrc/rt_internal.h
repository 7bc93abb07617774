// Internal declarations shared by the library's translation units: kernel
// parameter blocks and the host-side launchers that dispatch on log2(n).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rtk {

// Device allocation used by the whole library (cudaMalloc), with the
// fault-injection hook behind rt_debug_fail_alloc.
cudaError_t dev_alloc(void **p, size_t bytes);
template <typename T> inline cudaError_t dev_alloc(T **p, size_t bytes)
{
    return dev_alloc(reinterpret_cast<void **>(p), bytes);
}

enum PumpKind { PUMP_SUPERGAUSS = 0, PUMP_UNIFORM = 1, PUMP_ARRAY = 2 };

// Pump evaluation inside the FP32 row sweep: super-Gaussian of order 10
// computed on the fly, uniform, or a precomputed N0 table (array pumps and
// any other super-Gaussian order).
enum PumpEval { PE_SG10 = 0, PE_UNIFORM = 1, PE_TABLE = 2, PE_RUNTIME = 3 /* chosen per call */ };

template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

// Local map parameters: E <- sqrtR * A * D * exp(N/2) * E',
// N <- N + (N0 - N (1 + I invIsat)) invT1, N0 = g0 * P(x, y) (or, with
// relax_exact, the rate equation solved over the bounce).  D is the complex
// aperture beyond the hard edge (smooth taper, curved mirror, roughness, eq.
// complex_aperture2): either separable, D = lens[x] lens[y], or a full table
// D = phase[y n + x]; neither pointer set means D = 1.
template <typename R>
struct GainParams {
    R sqrtR, invT1, invIsat, g0;
    R inv_rp2;          // 1 / r_p^2 (super-Gaussian)
    R half_order;       // order / 2
    int int_half_order; // > 0 when order/2 is that integer (product form)
    int edge;
    int pump_kind;
    const R *pump_tab;  // n*n N0 values when pump_kind == PUMP_ARRAY
    const typename cplx_of<R>::type *lens;   // n per-axis factors A(j) exp(-i c x_j^2), or null
    const typename cplx_of<R>::type *phase;  // n*n factors A(x) A(y) exp(-i (c (x^2 + y^2) + psi)), or null
    int relax_exact;                         // 1: exponential inversion update
};

// Per-bounce mean intensity: block partials, reduced by the last block to
// arrive (fixed order, so the result is deterministic).
struct StatParams {
    double *part;          // one partial per block of the reducing kernel
    unsigned int *count;   // arrival counter, reset by the last block
    double *hist;          // ring of hist_cap means (may be null when hist_cap == 0)
    long long hist_cap;
    long long *bounce;     // device bounce counter (slot index for hist)
    double *last_mean;     // mean intensity after the last bounce
    int *err;              // sticky error word (0 or RT_ENUMERIC)
};

struct PeakResult {
    double value;
    long long index;
};

// One resonator of a batched launch (device memory): its state, propagator
// table, local-map parameters and statistics.  st.part must hold one double
// per row group.  Items of a resonator whose bounce counter has reached
// `target` are skipped, so resonators with different remaining bounce counts
// can share launches.
struct BatchRes {
    float2 *E;
    float *N;
    const float2 *h;
    const CUtensorMap *tmap;  // column-tile tensor map of E (64-byte aligned, device memory)
    GainParams<float> g;
    int pe;                   // PumpEval
    int pad;
    long long target;         // stop once *st.bounce >= target
    StatParams st;
};

// Batched sweeps over nres resonators of side 2^logn (descriptors `res` in
// device memory); err receives RT_ETIMEOUT if a copy wait runs out.
cudaError_t launch_col_batch32(int logn, int colC, const BatchRes *res, int nres, const float2 *tw, int *err,
                               cudaStream_t s, int order = 0);
cudaError_t launch_row_batch32(int logn, const BatchRes *res, int nres, const float2 *tw, int *err, cudaStream_t s);
cudaError_t prepare_batch32(int logn, int colC, int order = 0);
int row_groups32(int logn);  // row groups per resonator of a batched row sweep

// One launch per sweep over size classes of uneven sides 128..2048
// (mix_supported): every item holds the same number of points, the column
// tile of side n is mix_col_tile(n) columns wide (the slots' tensor maps must
// use that width).
struct MixLaunch {
    int logn;
    const BatchRes *res;
    int nres;
    const float2 *tw;
};
bool mix_supported(int logn);
int mix_col_tile(int logn);
cudaError_t prepare_mixed32();
cudaError_t launch_col_mixed32(const MixLaunch *cls, int ncls, int *err, cudaStream_t s);
cudaError_t launch_row_mixed32(const MixLaunch *cls, int ncls, int *err, cudaStream_t s);

// ---- FP32 fused path: two sweeps per bounce --------------------------------
// Column sweep: per column, forward FFT, x h(my), inverse FFT (in place).
// tmap: the field's column-tile tensor map (make_col_tensor_map); err: the
// handle's sticky error word (set to RT_ETIMEOUT if a copy wait runs out).
cudaError_t launch_col_diffract32(int logn, int colC, float2 *E, const float2 *tw, const float2 *h, const void *tmap,
                                  int *err, cudaStream_t s, int order = 0);
// Radix orders (0 .. col_orders32 - 1) of the column sweep at tile width colC
// (0 if the width does not fit); order 0 is the built-in sequence.
int col_orders32(int logn, int colC);
// Pass-major twiddles of radix order `order` (twiddle_entries(log2 n) entries suffice).
cudaError_t launch_twiddles32(int n, int order, float2 *tw, cudaStream_t s);
// Encode the 128-byte tensor map of an n x n complex64 field for column
// tiles of colC columns (copy-engine loads of the column sweep).
cudaError_t make_col_tensor_map(void *map, float2 *E, int n, int colC);
// Row sweep: per row, forward FFT, x h(mx), inverse FFT, then the local map
// (gain, mirror phase, edge, inversion update) and the mean-intensity
// reduction.  pe selects how N0 is evaluated: 0 super-Gaussian of order 10
// on the fly, 1 uniform, 2 from GainParams::pump_tab.  The general form of
// the kernel (aperture table, exact relaxation) runs as feature_form(g) says.
cudaError_t launch_row_diffract_gain32(int logn, int pe, float2 *E, float *N, const float2 *tw, const float2 *h,
                                       const GainParams<float> &g, const StatParams &st, cudaStream_t s);
int row_blocks32(int logn);            // most blocks of a row sweep (size of StatParams::part)
// Set kernel attributes (shared-memory opt-in) of a bounce's kernels on the
// current device; done before capturing a bounce into a CUDA graph.
// feat: the FeatureForm of the row sweep's local map.
cudaError_t prepare_bounce32(int logn, int colC, int pe, int feat);
cudaError_t prepare_row32(int logn, int pe, int feat);
cudaError_t prepare_col32(int logn, int colC);
cudaError_t prepare_bounce64(int logn);
int col_tile_ok32(int logn, int colC); // 1 if that column tile width is instantiated and fits
int default_col_tile32(int logn);      // column tile width used when none is requested (tuned or built in)
int builtin_col_tile32(int logn);      // the built-in choice
int set_tuned_col_tile32(int logn, int colC);  // record a tuned width (0 clears); 1 on success
int tuned_col_tile32(int logn);        // tuned width or 0
int set_tuned_col_order32(int logn, int order);  // record a tuned radix order (0: built-in); 1 on success
int tuned_col_order32(int logn);       // tuned radix order or 0

// Plain diffraction of a copy of the field (intracavity readout): rows out
// of place (in -> out), then columns in place, each forward FFT, x h,
// inverse FFT; h from launch_prop32/64 for the distance wanted.
cudaError_t launch_row_diffract_plain32(int logn, const float2 *in, float2 *out, const float2 *tw, const float2 *h,
                                        cudaStream_t s);
cudaError_t launch_col_diffract_plain32(int logn, float2 *X, const float2 *tw, const float2 *h, cudaStream_t s);
cudaError_t launch_row_diffract_plain64(int logn, const double2 *in, double2 *out, const double2 *tw,
                                        const double2 *h, cudaStream_t s);
cudaError_t launch_col_diffract_plain64(int logn, double2 *X, const double2 *tw, const double2 *h, cudaStream_t s);
cudaError_t launch_prop32(int n, double alpha, float2 *h, cudaStream_t s);
cudaError_t launch_prop64(int n, double alpha, double2 *h, cudaStream_t s);

// Forward 2-D transform helpers (spectrum readout), FP32: rows out of place, columns in place.
cudaError_t launch_row_fft32(int logn, const float2 *in, float2 *out, const float2 *tw, int dir, cudaStream_t s);
cudaError_t launch_col_fft32(int logn, float2 *X, const float2 *tw, int dir, cudaStream_t s);

// ---- FP64 plain path: six unfused sweeps per bounce --------------------------
cudaError_t launch_row_fft64(int logn, const double2 *in, double2 *out, const double2 *tw, int dir,
                             cudaStream_t s);
cudaError_t launch_col_fft64(int logn, double2 *X, const double2 *tw, int dir, cudaStream_t s);
cudaError_t launch_mul_h64(int n, double2 *E, const double2 *h, cudaStream_t s);
cudaError_t launch_gain64(int n, double2 *E, double *N, const GainParams<double> &g, const StatParams &st,
                          cudaStream_t s);
int gain_blocks64(int n);

// ---- set-up kernels (FP64 arithmetic, stored in the path's precision) -------
// Entries of the pass-major twiddle table of a line FFT of length 2^logn.
int twiddle_entries(int logn);
// tw: pass-major twiddles (twiddle_entries(log2 n) entries); h: n per-axis propagator values.
cudaError_t launch_tables32(int n, double alpha, float2 *tw, float2 *h, cudaStream_t s);
cudaError_t launch_tables64(int n, double alpha, double2 *tw, double2 *h, cudaStream_t s);
cudaError_t launch_noise32(int n, unsigned long long seed, double amp, float2 *E, cudaStream_t s);
cudaError_t launch_noise64(int n, unsigned long long seed, double amp, double2 *E, cudaStream_t s);
// Complex aperture factors, FP64 arithmetic (eq. complex_aperture2, its
// phase conjugated like the propagator): A(x) A(y) exp(-i theta),
// theta = c (x^2 + y^2) + psi(x, y), c = (pi / (4 alpha)) (z / F), A the
// per-axis modulus (0 in the edge band, a sin^2 ramp of `taper` pixels, 1
// inside).  lens: the n per-axis factors A(j) exp(-i c x_j^2); phase: the
// n*n factors with psi (device array of n*n doubles, or null for psi = 0).
double lens_curvature(double alpha, double z_over_F);
cudaError_t launch_lens32(int n, double c, int edge, int taper, float2 *lens, cudaStream_t s);
cudaError_t launch_lens64(int n, double c, int edge, int taper, double2 *lens, cudaStream_t s);
cudaError_t launch_phase32(int n, double c, int edge, int taper, const double *psi, float2 *phase, cudaStream_t s);
cudaError_t launch_phase64(int n, double c, int edge, int taper, const double *psi, double2 *phase,
                           cudaStream_t s);

// Forms of the row sweep's local map: the plain form (flat, hard-edged
// mirror, Euler inversion step) and the general forms, which multiply by an
// aperture table (g.phase, else g.lens, which must then be set; a table of
// ones serves a flat mirror) with the Euler or the exact inversion update.
enum FeatureForm { FEAT_PLAIN = 0, FEAT_TABLE = 1, FEAT_TABLE_EXACT = 2 };
template <typename R> __host__ __device__ inline int feature_form(const GainParams<R> &g)
{
    return g.relax_exact ? FEAT_TABLE_EXACT : ((g.lens || g.phase) ? FEAT_TABLE : FEAT_PLAIN);
}
// Structured starting field (rt_set_field_pattern), FP64 arithmetic.
cudaError_t launch_pattern32(int n, int kind, int q, int alt, double w, double env, double curv, double amp,
                             float2 *E, cudaStream_t s);
cudaError_t launch_pattern64(int n, int kind, int q, int alt, double w, double env, double curv, double amp,
                             double2 *E, cudaStream_t s);
// N0 = g0 * P in FP64 (profile: device array of n*n doubles or null), stored as R.
cudaError_t launch_pump32(int n, int kind, double g0, double order, double radius, const double *profile,
                          float *out, cudaStream_t s);
cudaError_t launch_pump64(int n, int kind, double g0, double order, double radius, const double *profile,
                          double *out, cudaStream_t s);

// ---- spectrum readout ----------------------------------------------------------
cudaError_t launch_power32(int n, const float2 *X, float *S, cudaStream_t s);
cudaError_t launch_power64(int n, const double2 *X, double *S, cudaStream_t s);
// Folded-power argmax over a power spectrum S (float or double).
cudaError_t launch_peak32(int n, int ring, const float *S, double *part_val, long long *part_idx,
                          unsigned int *count, PeakResult *out, cudaStream_t s);
cudaError_t launch_peak64(int n, int ring, const double *S, double *part_val, long long *part_idx,
                          unsigned int *count, PeakResult *out, cudaStream_t s);
int peak_blocks(int n);

}  // namespace rtk
