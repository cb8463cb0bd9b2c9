/* pespace_gb300.h -- C ABI of the GB300 (sm_103a) library that evaluates the frequency-domain
 * Whittle log-likelihood of massive-black-hole-binary signals in the TDI A/E/T channels of
 * LISA-, Taiji- and TianQin-like detectors (arXiv:2602.12011, Sec. 2).
 *
 * Conventions shared by every call
 *   - Units: masses in solar masses, distances in Gpc, times in seconds, angles in radians,
 *     frequencies in Hz, strain and TDI outputs in fractional-frequency units.
 *   - Parameter vector theta[11] (PE_NPARAM), in this order:
 *       Mtot [Msun], q = m1/m2 >= 1, chi1, chi2 (aligned spins), dL [Gpc], iota, phi_c,
 *       lambda (ecliptic longitude), beta (ecliptic latitude), psi, t_c [s]
 *     (the eleven parameters of the paper's Table tab_pe_res, with q inverted to q >= 1).
 *   - Mode mask bits: 0x01 (2,2), 0x02 (2,1), 0x04 (3,3), 0x08 (3,2), 0x10 (4,4).
 *   - Frequency grid of a detector: f_k = k / T_obs for k = k0 .. k0 + nbins - 1 (Sec. 3.1:
 *     numpy.fft.rfftfreq bins truncated to a band).
 *   - Complex arrays are interleaved (re, im) doubles. Channel-major layouts: [3][nbins][2]
 *     for A, E, T in that order.
 *   - Pointers named "may be host or device" are classified with cudaPointerGetAttributes;
 *     host buffers are copied through the library, device buffers are used in place.
 *   - Every call is enqueued on the caller's CUDA stream (NULL = the legacy default stream).
 *     Device outputs are valid once that stream has been synchronised. When an output pointer
 *     is a host pointer the call synchronises the stream before it returns.
 *   - Errors are reported by the return status only; pe_last_error() gives a message for the
 *     calling thread. No call aborts the process or throws across the ABI.
 *   - A parameter sample outside the domain (non-finite component, q < 1, |chi| >= 1,
 *     dL <= 0, Mtot outside [1e3, 1e9] Msun) is not an error: its log-likelihood is -inf, its
 *     gradient is zero, and its bit in the optional status array is set.
 *   - The library owns all device scratch memory; it is allocated stream-ordered
 *     (cudaMallocAsync) inside each call and released on the same stream.
 */
#ifndef PESPACE_GB300_H
#define PESPACE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PE_NPARAM 11
#define PE_MODE_22 0x01u
#define PE_MODE_21 0x02u
#define PE_MODE_33 0x04u
#define PE_MODE_32 0x08u
#define PE_MODE_44 0x10u
#define PE_MODE_ALL 0x1Fu
/* Precision flag, OR-ed into the mode_mask of the forward entry points (pe_loglike_batch,
 * pe_loglike_batch_noalloc, pe_plan_create, pe_autotune, pe_signal_aet). Without it every step
 * runs in FP64. With it the TaylorF2 phase, its reduction to a fraction of a turn and every sum
 * across tiles stay FP64, while t_f, the orbit angles and the response geometry (orbit offsets,
 * link vectors, projections, sincs, third-spacecraft phases, TDI brackets) run on the FP32 pipe
 * in double-word arithmetic (~48-bit significands, ~1e-14 relative; t_f and the orbit angles in
 * FP64 where t_f lies more than 2^23 s, heliocentric, or 2^21 s, geocentric, from the origin).
 * It agrees with the FP64 path to far below the 1e-10 parity bar but not bit for bit; each
 * precision is bitwise batch-invariant by itself. pe_loglike_grad_batch, pe_hetero_create and
 * pe_surrogate_loglike_batch also take the flag (see there); pe_fisher and
 * pe_surrogate_mismatch are FP64 only and reject it. */
#define PE_PREC_MIXED 0x100u
/* Precision flag for the precision study, OR-ed into the same mode masks (not with PE_PREC_MIXED):
 * every step in FP32, including the TaylorF2 phase, t_f and frac(f t_c) -- the paper's float32
 * option for coarse work (Sec. 3.1, Fig. fig_cost). Its log L misses the 1e-10 parity bar by
 * orders of magnitude; it exists to measure that trade, not for inference. */
#define PE_PREC_FP32 0x200u

typedef enum {
  PE_OK = 0,
  PE_EINVAL = 1,   /* invalid argument (NULL handle, bad size, mode mask, grid mismatch) */
  PE_ENOMEM = 2,   /* device or host allocation failed */
  PE_ECUDA = 3,    /* a CUDA runtime call failed */
  PE_ETIMEOUT = 4, /* a bounded host wait gave up */
  PE_ESTATE = 5    /* call out of order (e.g. likelihood before data was set) */
} pe_status;

typedef enum { PE_ORBIT_HELIO = 0, PE_ORBIT_GEO = 1 } pe_orbit_kind;

/* Detector description (Sec. 2.1 response model; Sec. 3.2 orbits and noise).
 *   orbit        PE_ORBIT_HELIO: Keplerian heliocentric constellation to first order in the
 *                eccentricity (LISA, Taiji); PE_ORBIT_GEO: equilateral triangle of radius
 *                arm/sqrt(3) around a circular-orbit Earth (TianQin).
 *   tdi_gen      15 or 20: FD TDI generation 1.5 or 2.0 (Sec. 2.1, after Eq. eq_tf).
 *   psd_shaping  1: apply the LISA-type low/high-frequency shaping factors to the noise.
 *   arm_m        nominal arm length L [m]; alpha0_rad initial revolution angle around the Sun;
 *   cartwheel0_rad initial constellation orientation (heliocentric only);
 *   geo_period_s, geo_lon_rad, geo_lat_rad: TianQin constellation period and normal direction.
 *   oms_m_rtHz, acc_ms2_rtHz: optical-metrology and test-mass acceleration noise levels. */
typedef struct {
  int32_t orbit;
  int32_t tdi_gen;
  int32_t psd_shaping;
  int32_t reserved;
  double arm_m;
  double alpha0_rad;
  double cartwheel0_rad;
  double geo_period_s;
  double geo_lon_rad;
  double geo_lat_rad;
  double oms_m_rtHz;
  double acc_ms2_rtHz;
} pe_detector_config;

typedef struct pe_detector_s* pe_detector; /* opaque; owned by the library */

/* Create a detector on the current CUDA device with the grid f_k = k/T_obs,
 * k in [k0, k0 + nbins). Allocates the per-bin device tables (about 150 bytes per bin).
 * Errors: PE_EINVAL for a NULL cfg/out, nbins < 1, k0 < 1, T_obs <= 0, tdi_gen not 15/20,
 * orbit not 0/1, arm_m <= 0; PE_ENOMEM; PE_ECUDA. */
pe_status pe_create_detector(const pe_detector_config* cfg, double T_obs, int64_t k0, int64_t nbins,
                             pe_detector* out);

/* Free the detector and its device memory (synchronises the device first). NULL is a no-op. */
pe_status pe_destroy_detector(pe_detector det);

/* Analytic noise PSD of A, E, T on the detector grid (Sec. 3.2: acceleration + OMS noise only,
 * equal-arm TDI, times |1 - z^4|^2 for TDI 2.0). out_psd: HOST array [3][nbins]. */
pe_status pe_psd_model(pe_detector det, double* out_psd);

/* Set the data and PSD the likelihood uses (Eq. eq_ll_fd, Eq. eq_inner_product). The library
 * copies both, builds the whitened per-bin tables and <d|d> per channel.
 *   data_aet: [3][nbins][2] complex data d~_c(f_k) (host or device);
 *   psd_aet:  [3][nbins] one-sided PSD S_c(f_k) (host or device), or NULL for pe_psd_model's;
 *   ptr_is_device: 1 if both pointers are device pointers, 0 if host.
 * Synchronous. Errors: PE_EINVAL (NULL det/data, non-positive or non-finite PSD value). */
pe_status pe_set_data_psd(pe_detector det, const double* data_aet, const double* psd_aet, int ptr_is_device);

/* <d|d> per channel (after pe_set_data_psd). out_dd: host double[3]. */
pe_status pe_data_norm(pe_detector det, double* out_dd);

/* Noise-free signal h~_c(f_k) of one source in the A, E, T channels on the detector grid:
 * TaylorF2 modes (SPA, time-frequency map Eq. eq_tf), single-link response Eq. eq_fd_resp at
 * t_f, FD TDI and A/E/T (Sec. 2.1). theta: [11] (host or device); out: [3][nbins][2]
 * (host or device). Out-of-domain theta gives PE_EINVAL. mode_mask may carry PE_PREC_MIXED. */
pe_status pe_signal_aet(pe_detector det, const double* theta, unsigned mode_mask, double* out, void* stream);

/* Data = noise-free signal of theta_inj + noise with Re, Im ~ N(0, S_c T/4) (Eq.
 * eq_diag_Sigma_to_Sn), using the detector's analytic PSD, then pe_set_data_psd(data, NULL).
 * normals: HOST [3][nbins][2] standard-normal draws supplied by the caller, or NULL for
 * noise-free data. Synchronous. */
pe_status pe_inject(pe_detector det, const double* theta_inj, unsigned mode_mask, const double* normals);

/* Batched joint log-likelihood over ndet detectors and the A/E/T channels (Eq. eq_ll_fd with
 * the joint product over channels and detectors, Sec. 2.2):
 *   logL_s = sum_I sum_c ( <d|h>_{I,c} - 1/2 <h|h>_{I,c} - 1/2 <d|d>_{I,c} ).
 *   dets[ndet]: detector handles, each with data set; 1 <= ndet <= 8.
 *   theta: [B][11] (host or device), 1 <= B <= 1048576.
 *   out_logl: [B] (host or device).
 *   out_dhhh: nullable [B][ndet][3][2] = (<d|h>, <h|h>) per detector and channel.
 *   out_status: nullable int32 [B]; bit 0 = sample out of domain.
 *   mode_mask: PE_MODE_* bits (at least one), optionally | PE_PREC_MIXED.
 * Samples are independent: each sample's result depends only on its own theta (fixed-order
 * reductions), so it is identical in any batch. Errors: PE_EINVAL, PE_ESTATE, PE_ENOMEM, PE_ECUDA. */
pe_status pe_loglike_batch(const pe_detector* dets, int ndet, const double* theta, int B, unsigned mode_mask,
                           double* out_logl, double* out_dhhh, int32_t* out_status, void* stream);

/* pe_loglike_batch without any device allocation (the paper has no counterpart: this entry
 * point exists for callers that cannot allocate). A sampler embedded in an application that
 * reserves the GPU's memory for its own pool at start-up, or a latency-critical loop that must
 * never enter the allocator, cannot let the library call cudaMalloc/cudaMallocAsync per call.
 * This variant computes exactly what pe_loglike_batch computes (bit for bit), with its scratch in
 * one fixed 32 MiB device array; it calls no allocating routine.
 *   When the array is committed: CUDA loads the module that holds it lazily, on the first use of
 *   that module on a device -- the first pe_loglike_batch_noalloc call there. That call commits
 *   the 32 MiB (and can fail with PE_ECUDA if the device has no memory left); the device then holds
 *   it until the process exits. So make the first call on each device before the application
 *   reserves the device's memory for its own pool (and before any stream capture); every later
 *   call allocates nothing.
 *   theta, out_logl and the optional out_dhhh / out_status must be DEVICE pointers (host buffers
 *   would need staging memory); other arguments and layouts are as for pe_loglike_batch.
 *   Size limit: coefficients (1,136 bytes per sample) plus one 48-byte partial per 128-bin
 *   sub-tile of every (detector, sample) pair must fit in 32 MiB -- about 400 samples on one
 *   2^22 s grid (209,296 bins), about 1,500 on a 2^20 s grid, in every precision. Larger batches
 *   return PE_EINVAL with the needed size in pe_last_error(); split them. The work items take the
 *   precision's default sub-tile count (no tuned choice is read).
 *   Every call looks up the array's device address on the current device (cudaGetSymbolAddress;
 *   nothing is allocated once the module is loaded, and no address outlives a device reset).
 *   Device pointers must belong to the current device (PE_EINVAL otherwise).
 *   All calls share the one array: calls whose work overlaps on the GPU (other streams, other
 *   host threads) race on it and give wrong results; serialise them. Every scratch element is
 *   written before it is read within a call, so nothing is cleared between calls. */
pe_status pe_loglike_batch_noalloc(const pe_detector* dets, int ndet, const double* theta, int B, unsigned mode_mask,
                                   double* out_logl, double* out_dhhh, int32_t* out_status, void* stream);

/* ---- Uneven-batch plans and the autotuner (batched uneven launches) -------------------------
 * A plan is the whole pe_loglike_batch computation for fixed detectors, batch size, mode mask
 * and fixed DEVICE buffers (theta [B][11], out_logl [B], optional out_dhhh [B][ndet][3][2] and
 * out_status [B]), captured once into a CUDA graph with its scratch allocated at creation. Every
 * (detector, sample) pair brings its own grid length and active bin range; all pairs run in one
 * persistent launch over their bin tiles. Refill theta in place and call pe_plan_launch on
 * any stream; results equal pe_loglike_batch's bit for bit.
 *   The forward kernel's work items are 1, 2, 4 or 8 consecutive 128-bin sub-tiles of one
 *   (detector, sample) pair; each sub-tile keeps its own partial sum in a fixed reduction order.
 *   autotune = 1: if the tuning cache has no entry for this workload (GPU, SM count, batch size,
 *   mode mask, grids), time the forward kernel's launch choices on the theta present at
 *   creation (register-budget variant x persistent grid size, then the sub-tiles per work item)
 *   and store the fastest. The cache is a JSON file at $PE_TUNE_CACHE, else
 *   $XDG_CACHE_HOME/pespace_gb300/tune.json, else ~/.cache/pespace_gb300/tune.json.
 *   No choice changes a result (every choice keeps the same per-sub-tile partials). pe_loglike_batch
 *   also uses a cached choice.
 * pe_plan_info: the plan's choice (subtiles: sub-tiles per work item); tuned_ms 0 for a default.
 * pe_autotune tunes (and caches) the same choice without building a plan (theta: device).
 * pe_tune_set records a choice for a workload as the autotuner would (fwd_variant 0..2,
 *   ctas_per_sm 1..64, subtiles 1, 2, 4 or 8; PE_EINVAL otherwise); later calls and plans for
 *   that workload use it. */
typedef struct pe_plan_s* pe_plan;
pe_status pe_plan_create(const pe_detector* dets, int ndet, int B, unsigned mode_mask, const double* theta_dev,
                         double* out_logl_dev, double* out_dhhh_dev, int32_t* out_status_dev, int autotune,
                         pe_plan* out);
pe_status pe_plan_launch(pe_plan plan, void* stream);
pe_status pe_plan_info(pe_plan plan, int* fwd_variant, int* ctas_per_sm, int* subtiles, double* tuned_ms);
pe_status pe_plan_destroy(pe_plan plan);
pe_status pe_autotune(const pe_detector* dets, int ndet, const double* theta_dev, int B, unsigned mode_mask,
                      int* out_variant, int* out_ctas_per_sm, int* out_subtiles, double* out_ms);
pe_status pe_tune_set(const pe_detector* dets, int ndet, int B, unsigned mode_mask, int fwd_variant, int ctas_per_sm,
                      int subtiles);

/* ---- Learned waveform surrogate (MLP on BF16 tensor cores + node spline) ----------------------
 * An MLP 11 -> 256 -> 256 -> 256 -> 2560 (BF16 weights and activations on tensor cores, FP32
 * accumulation, SiLU) maps theta to, per mode, a phase residual and an amplitude ratio at 256
 * frequency nodes log-spaced from 1e-4 Hz to the mode's taper end m F_isco. The phase residual is
 * the plain generator's 3PN and 3.5PN phase terms (the series through 2.5PN, spins included, is
 * evaluated exactly at the nodes as the baseline), the
 * amplitude ratio its |H_lm| relative to the Newtonian power law. At the nodes the full response
 * (t_f, orbit, links, TDI) is evaluated in FP64 and not-a-knot cubic splines in ln f carry the
 * mode phase and the A/E/T transfer functions to every bin (the sparse-node interpolation idea the
 * paper cites for lisabeta, Sec. 1). Samples outside the training box, and detectors on a
 * geocentric orbit, take the plain path.
 *   pe_surrogate_create: random initial weights (seed); the library owns all device memory.
 *   pe_surrogate_train: trains on the plain generator's node values of theta_train_dev
 *     [n_train][11] (device) with Adam, MSE on standardised outputs, cosine learning rate, batch
 *     % 64 == 0; out_loss_curve (host, nullable) receives the last minibatch loss of each epoch.
 *   pe_surrogate_set_node_source: 0 (default) the network's node values; 1 the plain generator's
 *     own node values (the same spline path without the network, for comparison).
 *   pe_surrogate_set_box: the box of the node-spline path (defaults 1e5-1e7 Msun, q <= 10,
 *     |chi| <= 0.99: the prior's range); samples outside it take the plain path.
 *   pe_surrogate_set_network_qmax: the largest mass ratio whose node values come from the network
 *     (default 8: where the held-out mismatch of the trained network stays <= 1e-3); in-box samples
 *     above it take the plain generator's own node values on the same spline path. q_net >= 1.
 *   pe_surrogate_targets / pe_surrogate_predict: plain-generator / network node values
 *     [B][5][2][256] (fp32, device) for theta [B][11] (device).
 *   pe_surrogate_loglike_batch: log L per sample through the surrogate path (device pointers);
 *     out_used_dev (nullable) = 1 where the surrogate was used, 0 where the plain path was. A
 *     detector on a geocentric orbit (TianQin) always takes the plain path: its response turns
 *     too fast in t_f for the log-spaced nodes; used = 1 means the node splines served at least
 *     one heliocentric detector.
 *     mode_mask may carry PE_PREC_MIXED: out-of-box samples then take the mixed-precision plain
 *     path (as pe_loglike_batch with the flag) and in-box samples evaluate the spline phase in
 *     FP64, its sine and cosine and the transfer functions on the FP32 pipe; A/E/T and the
 *     weighted per-bin products of both are double words. PE_PREC_FP32 gives PE_EINVAL.
 *   pe_surrogate_mismatch: 1 - <h_s|h_p>/sqrt(<h_s|h_s><h_p|h_p>) between the surrogate and the
 *     plain A/E/T signals on one detector (noise-weighted inner product, Eq. eq_inner_product;
 *     App. A's mismatch without the maximisation over t_c and phi_c); 0 for fallback samples.
 *     FP64 only: a precision flag in mode_mask gives PE_EINVAL.
 *   pe_surrogate_mlp_debug / pe_surrogate_get_weights: forward + backward of the network on given
 *     inputs and output cotangents, and its weights, for gradient checks.
 *   pe_surrogate_mlp_trace: pe_surrogate_mlp_debug that also copies every intermediate of the pass
 *     to the host buffer trace (float32, B * 6464 values; bf16 buffers widened exactly), in this
 *     order, each [B][n] row-major: X (n = 64, the bf16 input features); for layer l = 0, 1, 2
 *     Z_l (256, fp32 pre-activation) then H_l (256, bf16 SiLU output); Y (2560, fp32); then for
 *     l = 2, 1, 0: dH_l (256, fp32 cotangent of H_l), dZ_l (256, fp32) and its bf16 copy (256).
 *     For elementwise checks of each layer against its own inputs; x, dy, y, grads as above.
 *   pe_surrogate_save / pe_surrogate_load: versioned binary checkpoint (weights, Adam state,
 *     output standardisation, box and network bound, seed) with an FNV-1a checksum; PE_EINVAL on a
 *     bad file. */
typedef struct pe_surrogate_s* pe_surrogate;
pe_status pe_surrogate_create(uint64_t seed, pe_surrogate* out);
pe_status pe_surrogate_destroy(pe_surrogate s);
pe_status pe_surrogate_train(pe_surrogate s, const double* theta_train_dev, int n_train, int epochs, int batch,
                             double lr, double* out_final_loss, float* out_loss_curve);
pe_status pe_surrogate_set_box(pe_surrogate s, double mtot_lo, double mtot_hi, double q_max, double chi_max);
pe_status pe_surrogate_set_node_source(pe_surrogate s, int source);
pe_status pe_surrogate_set_network_qmax(pe_surrogate s, double q_net);
pe_status pe_surrogate_targets(const double* theta_dev, int B, float* out_dev);
pe_status pe_surrogate_predict(pe_surrogate s, const double* theta_dev, int B, float* out_dev);
pe_status pe_surrogate_loglike_batch(pe_surrogate s, const pe_detector* dets, int ndet, const double* theta_dev, int B,
                                     unsigned mode_mask, double* out_logl_dev, int32_t* out_used_dev, void* stream);
pe_status pe_surrogate_mismatch(pe_surrogate s, pe_detector det, const double* theta_dev, int B, unsigned mode_mask,
                                double* out_mismatch_dev, void* stream);
pe_status pe_surrogate_mlp_debug(pe_surrogate s, const float* x, int B, const float* dy, float* y, float* grads);
pe_status pe_surrogate_mlp_trace(pe_surrogate s, const float* x, int B, const float* dy, float* y, float* grads,
                                 float* trace);
pe_status pe_surrogate_get_weights(pe_surrogate s, float* out, int64_t* count);
pe_status pe_surrogate_save(pe_surrogate s, const char* path);
pe_status pe_surrogate_load(pe_surrogate s, const char* path);

/* Batched gradient d logL_s / d theta_s (hand-written adjoint of the same path, Sec. 2.3 on
 * automatic differentiation); arguments as pe_loglike_batch, plus out_grad [B][11]
 * (host or device). out_logl may be NULL. mode_mask may carry PE_PREC_MIXED: the per-bin
 * forward mode sum (which out_logl and the cotangents come from) then runs in the mixed-precision
 * unit of pe_loglike_batch, and the reverse sweeps keep FP64 for the phase, t_f, the turn
 * reductions, the PN-coefficient chain rule and the sums, with the geometry, link factors and
 * their cotangents in double words. PE_PREC_FP32 gives PE_EINVAL. */
pe_status pe_loglike_grad_batch(const pe_detector* dets, int ndet, const double* theta, int B, unsigned mode_mask,
                                double* out_logl, double* out_grad, int32_t* out_status, void* stream);

/* Fisher matrix F_ij = <d h/d theta_i | d h/d theta_j> summed over detectors and channels
 * (Sec. 2.2, the equation after Eq. eq_ll_fisher), for B parameter points.
 * theta: [B][11] (host or device); out_F: [B][11][11] row-major (host or device). */
pe_status pe_fisher(const pe_detector* dets, int ndet, const double* theta, int B, unsigned mode_mask,
                    double* out_F, void* stream);

/* ---- Measurement helpers (no counterpart in the paper; used by the benchmark) ----------------
 * pe_profile_enable(1) makes the library record a CUDA event pair, on the call's stream, around
 * every launch of its fused per-bin kernels (log-likelihood forward, gradient, Fisher);
 * pe_profile_read waits for those events, returns the summed device time [ms] and the number of
 * launches since the previous read, and clears the record. pe_profile_enable(0) stops recording.
 * pe_measure_fp64_peak runs an FP64 fused-multiply-add throughput kernel (8 independent chains
 * per thread, one grid of 8 CTAs of 256 threads per SM) for about `seconds` and returns the
 * achieved FP64 rate in TFLOP/s (one FMA = 2 flops): the ALU roofline of the FP64 kernels.
 * pe_measure_fp32_peak does the same with FP32 FMAs: the FP32-pipe roofline of the double-word
 * arithmetic of the mixed-precision path (PE_PREC_MIXED). */
pe_status pe_profile_enable(int on);
pe_status pe_profile_read(double* total_ms, int64_t* launches);
pe_status pe_measure_fp64_peak(double seconds, double* out_tflops);
pe_status pe_measure_fp32_peak(double seconds, double* out_tflops);

/* Fisher-Gaussian approximation of the posterior on a subset of the parameters (Sec. 2.2: the
 * high-SNR likelihood Eq. eq_ll_fisher with covariance C = F^-1; Sec. 3.3 applies it to lambda,
 * beta, psi, t_c with the other parameters held at their fiducial values). Computes the full
 * Fisher matrix at theta0 (host [11]) with pe_fisher, takes the sub-block on idx[k] (host, distinct
 * indices in [0, 11)), inverts it by Cholesky, and maps the caller's standard normals
 * normals[n][k] (host) to samples out_samples[n][11] (host) = theta0 + L z with C = L L^T (other
 * components equal theta0). out_cov: host [k][k]. n may be 0 (then normals/out_samples may be
 * NULL). PE_EINVAL if the sub-block is not positive definite. Synchronous. */
pe_status pe_fisher_gaussian(const pe_detector* dets, int ndet, const double* theta0, unsigned mode_mask,
                             const int32_t* idx, int k, const double* normals, int n, double* out_cov,
                             double* out_samples);

/* ---- Heterodyned (relative-binning) likelihood (Sec. 1: heterodyning about a reference signal) ----
 * Relative to a reference theta0 near the truth, each mode's channel signal is h0 times a ratio
 * r = h(theta)/h0 that varies slowly with frequency. Inside coarse bin b = [f_b, f_b+1) the ratio is
 * linear, r0 + r1 (f - f_b), from its values at the edges. Data and reference enter through
 * per-bin summary sums over the fine grid, formed once at creation:
 *   A_o = sum_k w conj(d) h0_lm (f - f_b)^o,           o = 0, 1
 *   B_o = sum_k w h0_lm conj(h0_l'm') (f - f_b)^o,     o = 0, 1, 2
 * per mode (pair) and channel. A sample then needs the response only at the NE edges, not at
 * every bin: <d|h> = sum Re[A0 r0 + A1 r1] and
 * <h|h> = sum Re[B0 r0 r0'* + B1 (r1 r0'* + r0 r1'*) + B2 r1 r1'*], with <d|d> exact.
 * Ratio rule: past a mode's last taper mark (1 - 0.1 * 0.7^10 of m F_isco, weight ~1e-15) and
 * wherever h0 is exactly zero, the previous edge's ratio is carried forward.
 *   pe_hetero_default_edges: host only, no GPU. Coarse edges (fine-bin indices, 0 .. kmax, kmax = the
 *     last bin below the reference's band end) for a grid (T_obs, k0, nbins) and theta0 [11] (host):
 *     nbins_coarse steps uniform in the relative-binning phase metric
 *     sum_g sgn(g) (f/f*_g)^g, g in {-5/3, -2/3, 1, 5/3, 7/3}, snapped to the grid, plus 11
 *     geometric marks 1 - 0.1 * 0.7^j (j = 0..10) of each mode's taper end; none past a mode's last
 *     mark inside its band. *inout_n: capacity of out_edges on entry, count on return (PE_EINVAL
 *     if too small).
 *   pe_hetero_create: summary data for detector det (with data set), reference theta0 [11] (host),
 *     mode_mask and edges [nedges] (host, strictly increasing, 2 <= nedges <= 640, within the grid).
 *     mode_mask may carry PE_PREC_MIXED: pe_hetero_loglike_batch then evaluates the signal at the
 *     edges with the mixed-precision unit and the per-bin contraction in double words (the
 *     summary data are built in FP64, the sums across bins stay FP64). An edge where a ratio
 *     h/h0 reaches 2^24 (a reference that has almost vanished, e.g. past its taper) keeps FP64
 *     ratios, and the bins that read it are contracted in FP64. PE_PREC_FP32 gives PE_EINVAL.
 *     The library owns the result; det must outlive it. Synchronous.
 *   pe_hetero_loglike_batch: log L per sample for hets[ndet] (1..8 detectors sharing one mode mask),
 *     theta [B][11], out_logl [B], out_dhhh nullable [B][ndet][3][2], out_status nullable [B] (host or
 *     device each, as pe_loglike_batch). One CTA per sample evaluates all NE edges of every detector.
 *   The heterodyned log L equals the exact one at theta0 and for changes of d_L or phi_c; elsewhere
 *   its error shrinks as the bins do (tests/test_gpu_hetero.py measures it). */
typedef struct pe_hetero_s* pe_hetero;
pe_status pe_hetero_default_edges(double T_obs, int64_t k0, int64_t nbins, const double* theta0, unsigned mode_mask,
                                  int nbins_coarse, int64_t* out_edges, int* inout_n);
pe_status pe_hetero_create(pe_detector det, const double* theta0, unsigned mode_mask, const int64_t* edges,
                           int nedges, pe_hetero* out);
pe_status pe_hetero_loglike_batch(const pe_hetero* hets, int ndet, const double* theta, int B, double* out_logl,
                                  double* out_dhhh, int32_t* out_status, void* stream);
pe_status pe_hetero_destroy(pe_hetero h);

/* Bounded host waits. An entry point that returns results into host memory waits for its stream
 * by polling an event (no blocking synchronise), for at most the limit set here (seconds, default
 * 600, process-wide). Past the limit it returns PE_ETIMEOUT: the work stays queued on the stream and
 * the host outputs are valid only once the stream has finished (cudaStreamSynchronize, or a later
 * wait). No counterpart in the paper. pe_set_wait_limit: PE_EINVAL unless 0 < seconds < inf. */
pe_status pe_set_wait_limit(double seconds);
double pe_get_wait_limit(void);

/* Message describing the last failing call on this thread ("" if none). */
const char* pe_last_error(void);

/* Library ABI version (increments on incompatible change). */
int pe_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PESPACE_GB300_H */
