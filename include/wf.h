/*
 * wf.h — C ABI of the GB300 messenger-field Wiener filter and Wiener-posterior sampler.
 *
 * Problem (Jeffrey, Heavens & Fortio, "Fast Sampling from Wiener Posteriors for Image Data with
 * Dataflow Engines", §1.1 Eq. 1-3 and §2.1 Eq. 4): data d = s + n on an H x W image (A = I), signal
 * covariance S diagonal in Fourier space with power spectrum P(k) (§2.1, Eq. 7), noise covariance N
 * diagonal in pixel space, missing pixels = infinite noise (§1.1). The library computes
 *   - wf_solve:  the Wiener filter s_W = S (S + N)^-1 d (Eq. 2-3) by the G -> 0 messenger iteration
 *                with lambda-cooling (§2.2, text after Alg. 1);
 *   - wf_sample: draws from the Wiener posterior (Eq. 4) by the messenger-field Gibbs sampler (Alg. 1).
 *
 * Conventions (all calls):
 *   - d, Ndiag: float32 [H][W], row-major. Ndiag > 0 is the noise variance; both are ignored where
 *     mask != 0.
 *   - mask: uint8 [H][W], nonzero = missing pixel.
 *   - Pk: float32 [H][W/2+1], the half spectrum (ky in FFT order 0..H-1, kx = 0..W/2): P_k is the
 *     variance of the unitary 2D DFT coefficient of s at mode k, i.e. <|(U s)_k|^2> with
 *     U = F / sqrt(H W) and F the transform of Eq. 6 (the paper's unnormalised F has variance H W P_k).
 *     P_k >= 0; P_k must be symmetric under k -> -k for the edge columns kx = 0 and kx = W/2.
 *   - tau: messenger variance T = tau I (Alg. 1 definitions). tau <= 0 selects the paper's choice,
 *     the minimum observed Ndiag (max_k P_k if every pixel is missing). A tau above the minimum observed
 *     Ndiag is rejected with WF_ERR_TAU.
 *   - Supported sizes: H == W in {16, 32, 64, 128, 256, 512, 1024} (wf_supported_size). Up to 128 x 128
 *     a chain's field stays in one SM's shared memory for the whole call. At 256 x 256 and 512 x 512 the
 *     samplers and Wiener filters of many chains or images keep each field in the shared memory of one
 *     thread-block cluster (wf_set_large_image_sampler). Otherwise larger images keep the field in global
 *     memory and run as
 *     one cooperative launch (all CTAs co-resident) whose phases are separated by a bounded grid barrier
 *     (WF_ERR_TIMEOUT if a barrier wait gives up). For those sizes wf_solve_ex starts from zero
 *     (opts->init_s must be NULL).
 *   - Pointers named d, Ndiag, mask, Pk, out*, init_s are DEVICE pointers owned by the caller; pointers
 *     to iters_out / resid_out / opts are HOST pointers (may be NULL where stated).
 *   - The sample outputs of wf_sample, wf_sample_ex, wf_sample_band and wf_sample_spin2 (out, out_P)
 *     may instead be page-locked host memory mapped into the device address space at the same address
 *     (cudaHostAlloc, or cudaHostRegister with mapping, under unified addressing); the kernel then
 *     stores each sample straight into host memory over the CPU-GPU link, with no staging buffer or
 *     copy. Page-locked memory without that mapping, or pageable host memory on a device that cannot
 *     access it (cudaDevAttrPageableMemoryAccess = 0), is refused with WF_ERR_ARG.
 *   - Calls are ordered on `stream` and return after the stream has reached their end (they
 *     synchronise on it to read the device status). The library allocates its scratch with
 *     cudaMallocAsync on `stream` and frees it before returning.
 *   - Errors never abort: the return value says what went wrong; outputs are then unspecified.
 *     WF_ERR_CUDA keeps the CUDA error code for wf_last_cuda_error().
 */
#ifndef WF_H_
#define WF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* wf_stream_t; /* binary-compatible with cudaStream_t; NULL = legacy default */

typedef enum {
  WF_OK = 0,
  WF_ERR_ARG = 1,            /* bad pointer / count / option, or Ndiag <= 0 / P < 0 on the inputs */
  WF_ERR_TAU = 2,            /* tau > min observed Ndiag */
  WF_ERR_SHAPE = 3,          /* unsupported H, W */
  WF_ERR_CUDA = 4,           /* a CUDA runtime call failed: see wf_last_cuda_error() */
  WF_ERR_NOT_CONVERGED = 5,  /* wf_solve reached max_iter; the last iterate is written */
  WF_ERR_NONFINITE = 6,      /* NaN/Inf in an observed input, in P, or in the residual */
  WF_ERR_TIMEOUT = 7         /* reserved: a bounded device-side wait gave up */
} wf_status;

/* Options of the Wiener-filter solve (wf_solve_ex). Fill with wf_solve_opts_default first. */
typedef struct {
  double tau;        /* <= 0: minimum observed Ndiag (Alg. 1 definition of T) */
  double tol;        /* stop when the lambda = 1 relative residual ||s + S N^-1 (s - d)|| / ||S N^-1 d|| < tol */
  double eta;        /* cooling factor in (0, 1): lambda_{j+1} = max(1, eta lambda_j), lambda_0 = max(1, max P / tau) */
  double level_tol;  /* a level lambda > 1 ends when its own relative residual < level_tol ... */
  int32_t level_max; /* ... or after level_max sweeps at that level */
  int32_t check;     /* residual measured every `check` sweeps (>= 1) */
  int32_t max_iter;  /* sweep budget of each messenger solve; WF_ERR_NOT_CONVERGED when exhausted */
  int32_t refine;    /* k > 0 (default 3): up to k mixed-precision refinement steps. The FP32 messenger
                        solve stops at max(tol, 1e-5); then the residual r = N^-1 (d - s) - S^-1 s of the
                        map and the stopping test are evaluated in FP64 on the GPU, and each step adds the
                        FP32 messenger solution e of (S^-1 + N^-1) e = r. resid_out is then the FP64
                        relative residual of the returned map, and WF_ERR_NOT_CONVERGED means it is still
                        >= tol after k steps. 0: the plain FP32 iteration to tol; resid_out is then its
                        own estimate from two consecutive FP32 iterates, which keeps falling below the
                        FP32 floor (the true residual of the map plateaus near 2e-6) */
  const float* init_s; /* device [H][W] starting iterate, or NULL for zero (sizes <= 128 only) */
  double refine_tol; /* relative residual target of each correction solve */
  const float* A;    /* device [H][W] diagonal pixel response of d = A s + n (Eq. 1), or NULL for A = I.
                        Pixels with A = 0 carry no data. tau (default) = min over data pixels of
                        Ndiag / A^2 (Alg. 1 definition of T). Solved as the same problem with data d / A
                        and noise Ndiag / A^2, which the t-update of Alg. 1 with A_i^2 > 0 equals exactly */
} wf_solve_opts;

/* Options of the sampler (wf_sample_ex). Fill with wf_sample_opts_default first. */
typedef struct {
  double tau;            /* <= 0: minimum observed Ndiag */
  int64_t n_samples;     /* samples kept per chain (>= 0) */
  int32_t n_chains;      /* independent chains (>= 1), all for the same data */
  uint32_t chain_offset; /* chain c uses Philox chain word chain_offset + c */
  uint32_t start_step;   /* Philox step word of the first sweep (resume a chain exactly) */
  int32_t burn_in;       /* sweeps discarded before the first kept sample (>= 0) */
  int32_t thin;          /* sweeps between kept samples (>= 1) */
  int32_t init_per_chain;/* 1: init_s is [n_chains][H][W]; 0: one [H][W] state shared by all chains */
  const float* init_s;   /* device starting state(s), or NULL for zero */
  const float* A;        /* device [H][W] diagonal pixel response (as wf_solve_opts::A), or NULL for A = I;
                            not accepted by wf_sample_noalloc (WF_ERR_ARG) */
  int32_t out_dtype;     /* element type of `out`: WF_OUT_F32 (default), or the FP32 state rounded once to
                            nearest even as WF_OUT_BF16 or WF_OUT_F16 (2 bytes per value; `out` then points
                            to such elements). The chain itself always runs in FP32. */
} wf_sample_opts;

#define WF_OUT_F32 0
#define WF_OUT_BF16 1
#define WF_OUT_F16 2

void wf_solve_opts_default(wf_solve_opts* o);
void wf_sample_opts_default(wf_sample_opts* o);

/*
 * Wiener filter (Eq. 2-3) by the G -> 0 messenger iteration with lambda-cooling (§2.2).
 * out_s: device float32 [H][W]. iters_out (host, may be NULL): sweeps performed (all solves).
 * resid_out (host, may be NULL): the relative residual ||s + S N^-1 (s - d)|| / ||S N^-1 d|| of the
 * returned map, summed in FP64 on the GPU (-1 if never measured). WF_OK means it is below tol.
 * Uses the defaults of wf_solve_opts_default (FP64-residual refinement, refine = 3) with the given tau
 * and tol.
 */
wf_status wf_solve(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H,
                   int32_t W, double tau, double tol, float* out_s, int32_t* iters_out, double* resid_out,
                   wf_stream_t stream);

/* As wf_solve with every option explicit (opts may be NULL: defaults). */
wf_status wf_solve_ex(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H,
                      int32_t W, const wf_solve_opts* opts, float* out_s, int32_t* iters_out, double* resid_out,
                      wf_stream_t stream);

/*
 * Wiener-posterior samples (Eq. 4) by Algorithm 1: one chain from s_0 = 0, no burn-in, thin 1, chain
 * word 0, first step word 0. out: device float32 [n_samples][H][W]; sample m is the state after sweep
 * m + 1. G(0,1) variates come from Philox4x32-10 with key (seed low word, seed high word) and counter
 * (group, step, chain, stream). The messenger draw xi uses stream 0, group (y W + x) / 4 and variate
 * (y W + x) % 4. The signal draw zeta uses stream 1: for 0 < kx < W/2, group kx H/2 + j holds mode
 * (j, kx) in variates 0, 1 (Re, Im) and mode (H - j, kx) in variates 2, 3 (j = 0: modes 0 and H/2); in
 * the columns kx = 0 and kx = W/2, group j (0 < j < H/2) holds mode (j, 0) in variates 0, 1 and mode
 * (j, W/2) in variates 2, 3, their conjugates fill the rows H - j, and group 0 holds the four real modes
 * (0, 0), (H/2, 0), (0, W/2), (H/2, W/2). Complex modes are (Re + i Im) / sqrt(2). Draws are therefore
 * reproducible, and an FP64 implementation of the same layout reproduces them draw for draw.
 */
wf_status wf_sample(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H,
                    int32_t W, int64_t n_samples, uint64_t seed, float* out, wf_stream_t stream);

/*
 * Several chains, burn-in, thinning, resume. out: device float32 [n_chains][n_samples][H][W]; sample m of
 * chain c is the state after sweep burn_in + (m + 1) * thin of that chain; sweep i uses Philox step word
 * start_step + i and chain word chain_offset + c. Resuming from sample m with start_step advanced by
 * the sweeps done reproduces the uninterrupted chain exactly.
 */
wf_status wf_sample_ex(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H,
                       int32_t W, uint64_t seed, const wf_sample_opts* opts, float* out, wf_stream_t stream);

/*
 * Hierarchical Gibbs sampler (the power spectrum inference of §5): Alg. 1 sweeps alternated with draws of
 * a binned power spectrum. bins: device int32 [H][W/2+1], the bin in [0, n_bins) of each half-spectrum
 * mode, or -1 for modes whose power stays at Pk (for instance k = 0); the map must be symmetric under
 * k -> -k, as P is. P0: device float32 [n_bins], the initial band powers (>= 0). Each sweep runs the t-draw,
 * the s-draw with P_k = P_b(k), then the band draw P_b | s ~ InvGamma(n_b / 2, S_b / 2) (prior 1 / P_b),
 * with S_b the sum of |U s|^2 over the full-spectrum modes of bin b and n_b their number, drawn as
 * P_b = S_b / X_b where X_b sums n_b squared normals from Philox stream 6 in the counter layout of the
 * s-draw (a complex mode pair gives Re^2 + Im^2, a self-conjugate mode one square). out_P (device float32
 * [n_chains][n_samples][n_bins], may be NULL) receives the band powers of each kept sample (drawn in the
 * same sweep). opts and out as for wf_sample_ex (a pixel response opts->A included). Sizes up to
 * 512 x 512 (256 and 512: one thread-block cluster per chain, the cluster sampler of wf_sample_ex with the
 * band draw added; WF_ERR_CUDA with cudaErrorNotSupported where the device cannot host such a cluster);
 * 0 <= n_bins <= 256 (512 at 512 x 512). A bin outside [-1, n_bins) or a negative or non-finite P0:
 * WF_ERR_ARG. The band sums S_b and X_b are FP32 sums in a fixed order, so a repeated call is
 * bit-identical. Scratch: one statistics buffer of 8 bytes per half-spectrum mode for every chain (up to
 * 128 x 128) or for every resident cluster (256 and 512), allocated per call on `stream`.
 */
wf_status wf_sample_band(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, const int32_t* bins,
                         int32_t n_bins, const float* P0, int32_t H, int32_t W, uint64_t seed,
                         const wf_sample_opts* opts, float* out, float* out_P, wf_stream_t stream);

/*
 * Spin-2 (shear) sampler for a convergence signal (the mass mapping of §5): data are the two real shear
 * components d1, d2 (noise variances N1, N2, one mask); the signal is kappa = kappa_E + i kappa_B with E and
 * B power spectra PE, PB ([H][W/2+1] as Pk), seen through the Kaiser-Squires operator: in Fourier space
 * gamma1_hat = c kappa_E_hat - s kappa_B_hat, gamma2_hat = s kappa_E_hat + c kappa_B_hat with
 * (c, s) = (cos 2 phi, sin 2 phi), phi the angle of k = (kx, ky), and (c, s) = (1, 0) at k = 0 and on the
 * Nyquist row and column. Each sweep is Alg. 1 for the pair: a t-draw per component (xi from Philox
 * streams 0 and 8), then per mode the rotation into E and B, the scalar s-draw of each with its spectrum
 * (zeta_E stream 1, zeta_B stream 9, the counter layout of wf_sample), and the rotation back. tau = the
 * minimum observed noise variance of both components unless opts->tau > 0. out: device
 * [n_chains][n_samples][2][H][W] shear samples (element type opts->out_dtype); opts->init_s, when given,
 * is [2][H][W] (or [n_chains][2][H][W] with init_per_chain). Sizes up to 512 x 512 (256 and 512: both
 * components of a chain in one thread-block cluster of 32-row CTAs; WF_ERR_CUDA with
 * cudaErrorNotSupported where the device cannot host such a cluster). opts->A, when given, is one pixel
 * response for both components (as in wf_sample_ex: d_c = A gamma_c + n_c, A = 0 meaning no data).
 */
wf_status wf_sample_spin2(const float* d1, const float* d2, const float* N1, const float* N2, const uint8_t* mask,
                          const float* PE, const float* PB, int32_t H, int32_t W, uint64_t seed,
                          const wf_sample_opts* opts, float* out, wf_stream_t stream);

/*
 * Wiener filter of the shear pair (the mass-mapping filter of §5): the G -> 0 form of wf_sample_spin2's
 * sweep with lambda-cooling. Per level lambda (lambda_0 = max(1, max(PE, PB) / tau), then
 * max(1, eta lambda)): opts->level_max sweeps with T = lambda tau (N_bar = N - tau fixed), no draws; at
 * lambda = 1 the FP64 relative residual ||g + S N^-1 (g - d)|| / ||S N^-1 d|| (S the shear covariance of
 * the E/B spectra) is evaluated every opts->check sweeps until it is below opts->tol or opts->max_iter
 * sweeps have run (WF_ERR_NOT_CONVERGED). out: device [2][H][W]; iters_out, resid_out: HOST, may be NULL.
 * Sizes up to 512 x 512 (256 and 512 on wf_sample_spin2's thread-block clusters); opts may be NULL
 * (defaults); opts->A, when given, is one pixel response for both components (the filter and its residual
 * are those of the response problem); opts->refine and init_s are not used.
 */
wf_status wf_solve_spin2(const float* d1, const float* d2, const float* N1, const float* N2, const uint8_t* mask,
                         const float* PE, const float* PB, int32_t H, int32_t W, const wf_solve_opts* opts, float* out,
                         int32_t* iters_out, double* resid_out, wf_stream_t stream);

/*
 * Convergence from shear fields: kappa_E_hat = c gamma1_hat + s gamma2_hat, kappa_B_hat = -s gamma1_hat +
 * c gamma2_hat (the inverse of the rotation above), with FP64 transforms. gamma: device [n][2][H][W];
 * kappa: device [n][2][H][W] (E then B). Any supported size.
 */
wf_status wf_shear_to_convergence(const float* gamma, int64_t n, int32_t H, int32_t W, float* kappa,
                                  wf_stream_t stream);

/*
 * Batched form: many independent images of possibly different sizes, each with its own data, noise map,
 * mask, power spectrum and outputs. For every item the library computes the Wiener filter (as wf_solve_ex
 * with the options below, from zero) and then n_samples posterior samples of one chain started at the
 * Wiener filter (Alg. 1 from s_0 = s_W, no burn-in, thin 1, Philox key `seed`, chain word `chain`, step
 * words 0 .. n_samples-1). Chains are independent (§4.2 of the paper runs independent chains in parallel).
 *   - Images up to 128 x 128, per size (opts->small_path): by default in phases (per-image set-up and
 *     tables, the level norms, one CTA per image for the cooled solve, then the samplers with several
 *     images per CTA), or as one persistent launch in which every CTA keeps one image's field in shared
 *     memory and takes images from an atomic work counter. 256 x 256 and 512 x 512 images: one
 *     thread-block cluster per image runs its whole pipeline with the field in distributed shared memory;
 *     1024 x 1024 images, small chunks and devices without room for a cluster: one cooperative launch per
 *     chunk with the fields in global memory. The size classes and the chunks of the large classes run
 *     on their own streams (`large_streams` per large class) and overlap. All of it is ordered after the
 *     work already on `stream` and the call returns when everything has finished.
 *   - items: HOST array; the pointers inside are DEVICE pointers owned by the caller; out_wf may be NULL
 *     (then the filter is not written), out_samples may be NULL when n_samples == 0.
 *   - On return items[i].status / iters / resid hold each image's wf_status, solve sweeps and last
 *     measured residual. The return value is WF_OK if every item succeeded, else the status of the first
 *     failing item (argument and CUDA errors abort the call before any work).
 */
typedef struct {
  const float* d;
  const float* Ndiag;
  const uint8_t* mask;
  const float* Pk;
  int32_t H, W;
  float* out_wf;       /* device [H][W] or NULL */
  float* out_samples;  /* device [n_samples][H][W] or NULL */
  uint64_t seed;
  uint32_t chain;
  int32_t status;      /* out */
  int32_t iters;       /* out */
  int32_t reserved;
  double resid;        /* out */
} wf_batch_item;

typedef struct {
  double tau;          /* <= 0: each image's minimum observed Ndiag */
  double tol, eta, level_tol;
  int32_t level_max, check, max_iter;
  int32_t n_samples;   /* samples per image (>= 0) */
  int32_t large_streams; /* concurrent pipelines for images above 128 x 128 (>= 1) */
  int32_t small_grid_pct; /* launch shape: persistent CTAs of each size class up to 128 x 128, in percent of
                             the occupancy limit (1..100; 0 = 100) */
  int32_t large_grid_pct; /* launch shape: CTAs of each cooperative launch for larger images, in percent of
                             the co-resident limit (1..100; 0 = 100); smaller grids let pipelines overlap */
  int32_t small_path;  /* images up to 128 x 128: 0 (default) = phased: per-image set-up and tables, then one
                          launch of every image's solve (a CTA each) and one of every image's samples (as
                          many images per CTA as the single-image sampler puts chains); 1 = fused: one
                          persistent kernel per size whose CTAs take images from a work counter and run the
                          whole pipeline each (small_grid_pct applies) */
  int32_t large_cluster_rows; /* 512 x 512 images on thread-block clusters: rows of the field per CTA, 32
                                 (clusters of 16 CTAs, 2 per SM) or 64 (clusters of 8 CTAs, 1 per SM);
                                 0 = 32 */
  int32_t small_fields_per_cta; /* phased path: images per CTA of the sampler launch of each size class up
                                   to 128 x 128, 1, 2, 4 or 8, capped at 128 / H (128 threads per CTA);
                                   0 = the cap */
} wf_batch_opts;

void wf_batch_opts_default(wf_batch_opts* o);
wf_status wf_batch_run(wf_batch_item* items, int32_t n_items, const wf_batch_opts* opts, wf_stream_t stream);

/*
 * The batched form recorded once as a CUDA graph and replayed. wf_batch_graph_create validates the items
 * and options exactly as wf_batch_run, allocates the batch's scratch for the graph's lifetime (device
 * memory, freed by wf_batch_graph_destroy), uploads the item table and captures the whole batch -- the
 * resets of the work counters and statuses, the launches of every size class up to 128 x 128 (phased or
 * fused, small_path) and the pipelines of the larger images, forked over streams and joined -- into one graph.
 *   - wf_batch_graph_launch enqueues one replay on `stream` and returns without waiting. Every replay
 *     recomputes every item from its inputs as they are in device memory when it runs (the pointers are
 *     fixed at creation). Replays share the graph's scratch: launch them on one stream (or order them).
 *   - wf_batch_graph_results waits for `stream` and copies each item's status, iters and resid of the last
 *     finished replay into items[0 .. n_items-1] (n_items must equal the created count); its return value
 *     is that of wf_batch_run.
 *   - creation runs a stream capture on a private stream; the device current at creation must be current
 *     for the other calls.
 */
typedef struct wf_batch_graph_s* wf_batch_graph;
wf_status wf_batch_graph_create(const wf_batch_item* items, int32_t n_items, const wf_batch_opts* opts,
                                wf_batch_graph* out);
wf_status wf_batch_graph_launch(wf_batch_graph g, wf_stream_t stream);
wf_status wf_batch_graph_results(wf_batch_graph g, wf_batch_item* items, int32_t n_items, wf_stream_t stream);
void wf_batch_graph_destroy(wf_batch_graph g);

/*
 * Launch-shape autotuner of the batched form. Starting from *opts, it times graph replays of this batch
 * (one warm-up and `reps` timed replays per candidate, CUDA events on `stream`) and keeps, one knob at a
 * time, the fastest large_grid_pct in {100, 50, 25, 12}, large_streams in {1, 2, 4, 8, 16} (when the batch has
 * images above 128 x 128), large_cluster_rows in {32, 64} (when it has 512 x 512 images), small_path in {0, 1}
 * and then, for the fused path, small_grid_pct in {100, 50, 25} or, for the phased path,
 * small_fields_per_cta in {1, 2, 4, 8} (when it has images up to 128 x 128); the chosen values are written
 * back to *opts and the
 * best replay time to *best_ms (HOST, may be NULL). The items' outputs are overwritten by the trial runs.
 * A representative subset of a large batch tunes faster than the whole batch.
 */
wf_status wf_batch_autotune(const wf_batch_item* items, int32_t n_items, wf_batch_opts* opts, int32_t reps,
                            double* best_ms, wf_stream_t stream);

/*
 * Weighted spectral power: out[f * nw + j] = sum_k w_j(k) |(U v_f)_k|^2 over the full spectrum, with
 * v_f = a_f + sgn * b_f (b may be NULL), U the unitary 2D DFT, f < n_fields, j < nw <= 4.
 * a, b: device float32 [n_fields][H][W]; w: device float32 [nw][H][W/2+1] (half-spectrum layout of Pk,
 * symmetric under k -> -k); out: HOST double [n_fields * nw]. (Building block of the gradient below;
 * S = U^dagger diag(P) U makes v^T S v the case w = P, §2.1 Eq. 7.)
 */
wf_status wf_spectral_power(const float* a, const float* b, float sgn, int32_t n_fields, const float* w, int32_t nw,
                            int32_t H, int32_t W, double* out, wf_stream_t stream);

/*
 * Gaussian log-likelihood of the data (§2.1: Gaussian likelihood and Gaussian-random-field prior,
 * A = I) for a power-law spectrum P(k) = amp (k/k0)^slope (P = 0 at k = 0, k in cycles/pixel as for Pk)
 * and noise N = alpha * sigma2, and its gradient with respect to (amp, slope, alpha):
 *   lnL = -1/2 d^T C^-1 d - 1/2 ln det C + const,  C = S + N over the observed pixels.
 * out_quad (HOST, may be NULL): Q = -1/2 d^T C^-1 d, exact up to the solve tolerance.
 * out_grad_quad (HOST double[3], may be NULL): dQ/dtheta = 1/2 x^T (dC/dtheta) x, x = C^-1 d, from one
 *   Wiener solve (x = N^-1 (d - s_W) on observed pixels) and weighted spectral powers of x.
 * out_grad (HOST double[3], may be NULL): d lnL / dtheta = dQ/dtheta - 1/2 tr(C^-1 dC/dtheta), the traces
 *   estimated with n_probes Rademacher probes z (Philox stream 5 keyed by seed; counter = (pixel/4,
 *   probe, 0, 5), sign from the top bit), each needing one more solve: C^-1 z = N^-1 (z - s_W(z)),
 *   run to max(tol, 1e-5) (far below the Monte-Carlo error of the estimate).
 * out_grad_var (HOST double[3], may be NULL): variance of the trace part of out_grad (sample variance
 *   over probes / n_probes).
 * out_wf (device [H][W], may be NULL): the Wiener filter of d.
 * d, sigma2: device float32 [H][W]; mask: device uint8 [H][W]; params = {amp, slope, k0, alpha}.
 */
wf_status wf_loglike_grad(const float* d, const float* sigma2, const uint8_t* mask, int32_t H, int32_t W,
                          const double* params, int32_t n_probes, uint64_t seed, double tol, double* out_quad,
                          double* out_grad_quad, double* out_grad, double* out_grad_var, float* out_wf,
                          wf_stream_t stream);

/*
 * wf_loglike_grad for many images at once: the forward Wiener solves of all images run as one batch
 * (wf_batch_run), then the probe solves of all images as a second batch. Each item's results equal those
 * of wf_loglike_grad with the item's own seed (same probes), up to the solve tolerance. Items are HOST
 * structs; d, sigma2, mask are device pointers ([H][W]); params = {amp, slope, k0, alpha}; the outputs
 * quad, grad_quad, grad (n_probes > 0) and grad_var are written into the items, with each item's status.
 * Returns WF_OK, or the first failing item's status (argument and CUDA errors before any work).
 */
typedef struct {
  const float* d;
  const float* sigma2;
  const uint8_t* mask;
  int32_t H, W;
  double params[4];
  uint64_t seed;
  double quad;          /* out */
  double grad_quad[3];  /* out */
  double grad[3];       /* out (n_probes > 0) */
  double grad_var[3];   /* out (n_probes > 0) */
  int32_t status;       /* out */
  int32_t reserved;
} wf_lik_item;

wf_status wf_loglike_grad_batch(wf_lik_item* items, int32_t n_items, int32_t n_probes, double tol,
                                wf_stream_t stream);

/*
 * The Wiener map (Eq. 2-3, A = I) as a function of the parameters of wf_loglike_grad (P = amp (k/k0)^slope,
 * N = alpha * sigma2): s_W(theta) = S[:, o] C^-1 d_o with C = S_oo + N_oo over the observed pixels o, and
 * its vector-Jacobian product for a cotangent g:
 *   out_vjp[i] = g^T d s_W / d theta_i = g^T dS[:, o] x - y^T (dC/dtheta_i) x,  theta = (amp, slope, alpha),
 *   x = C^-1 d_o = N^-1 (d - s_W) on o,  y = C^-1 (S g)_o  (C is symmetric, so the adjoint of the solve
 *   is one more Wiener solve: y = N^-1 (S g - s_W(S g)) on o, with the Wiener filter of "data" S g).
 * The dS terms are cross spectral powers sum_k dP_k Re(conj(U a)_k (U b)_k), evaluated as in
 * wf_spectral_power; S g is applied with FP64 transforms.
 *   s_w_in: device [H][W], the Wiener filter of d for these parameters kept from an earlier call (the
 *           checkpointed forward solve), or NULL: it is solved here.
 *   g:      device [H][W] cotangent, or NULL: only the forward map is computed (out_vjp untouched).
 *   tol:    relative-residual target of each solve; below 1e-6 the solves use FP64-residual refinement.
 *   out_vjp: HOST double[3] (required when g is given); out_wf: device [H][W] receiving s_W, or NULL.
 * d, sigma2: device float32 [H][W]; mask: device uint8 [H][W]; params = {amp, slope, k0, alpha}.
 * Statuses as wf_solve_ex (WF_ERR_NOT_CONVERGED when a solve misses tol).
 */
wf_status wf_wiener_vjp(const float* d, const float* sigma2, const uint8_t* mask, int32_t H, int32_t W,
                        const double* params, const float* g, const float* s_w_in, double tol, double* out_vjp,
                        float* out_wf, wf_stream_t stream);

/*
 * Self-test of the bounded device-side wait used by the large-image kernels (the grid barrier between
 * their phases). It runs one cooperative launch of n_blocks CTAs (1 .. 1024) whose barrier waits for one
 * arrival more than the grid has, so every wait reaches its poll limit (about a second) and gives up. The
 * expected result is WF_ERR_TIMEOUT with the context intact (later calls work); WF_OK would mean the wait
 * did not give up. elapsed_ms (HOST, may be NULL): the launch's duration. The paper has no counterpart:
 * this exercises the failure path of the library's waits without faulting the GPU.
 */
wf_status wf_selftest_wait_timeout(int32_t n_blocks, double* elapsed_ms);

/*
 * FP32 fused multiply-add throughput of the current device, measured: the denominator of the FP32
 * roofline the transforms' 5 n log2 n flops per sweep are reported against (the paper's method has no
 * dense contraction, so its bound is the FP32 pipe, not the tensor cores). One launch fills every SM to
 * its occupancy limit with CTAs of 256 threads, each thread running 16 independent chains of `iters`
 * FMAs (paired = 0: scalar FFMA; paired = 1: the paired form, two FMAs per instruction), timed with CUDA
 * events on `stream`; the call waits for it. tflops_out (HOST, may be NULL): 2 x FMAs / time in TFLOP/s;
 * ms_out (HOST, may be NULL): the launch's duration. iters in 1 .. 2^40, else WF_ERR_ARG. Changes no
 * device setting. The paper has no counterpart: this is measurement infrastructure.
 */
wf_status wf_measure_fp32_peak(int32_t paired, int64_t iters, double* tflops_out, double* ms_out,
                               wf_stream_t stream);

/* 1 if (H, W) is supported by wf_solve / wf_sample, else 0. */
int32_t wf_supported_size(int32_t H, int32_t W);

/* Static description of a status code (never NULL). */
const char* wf_status_string(wf_status s);

/* The cudaError_t of the last WF_ERR_CUDA returned on this thread (0 if none). */
int32_t wf_last_cuda_error(void);

/*
 * Kernel timing for benchmarks. With timing enabled (per host thread), each wf_solve* / wf_sample* call
 * records CUDA events on its stream around its main kernel (the fused Gibbs / Wiener-filter kernel,
 * not the set-up kernels); wf_last_kernel_ms returns that duration in milliseconds for the last call on
 * this thread, or -1 if timing was off or the call failed before the kernel.
 */
void wf_set_kernel_timing(int32_t enable);
double wf_last_kernel_ms(void);

/*
 * Path for 256 x 256 and 512 x 512 images (wf_sample, wf_sample_ex, the first pass of wf_solve /
 * wf_solve_ex, and the large images of wf_batch_run and the batch graphs), per host thread. Two kernel
 * families compute the same chain and the same filter (the same draws and schedule; FP32 results agree to
 * rounding): thread-block clusters, each holding one chain's or image's field in distributed shared memory
 * (N / 64 or N / 32 CTAs; a batch image runs its level norms, cooled solve and samples in one cluster),
 * and the global-memory kernels (fields in global memory, cooperative launches with many CTAs per field).
 * mode 0 (default, automatic): clusters when a call holds at least 32 chains at 256 x 256 or 8 at
 * 512 x 512 (a batch chunk as many images) and the device can host the cluster, otherwise the
 * global-memory kernels, which are faster for few fields; mode 1: always the global-memory kernels;
 * mode 2: clusters wherever the device can host them. Returns the previous mode.
 */
int32_t wf_set_large_image_sampler(int32_t mode);

/*
 * wf_sample_ex without any device allocation. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate GPU memory at call time, for instance real-time loops that cannot wait on
 * the allocator's latency and synchronisation, or host applications whose device memory is all owned by
 * their own pool or fixed in advance. Arguments, results and statuses are those of wf_sample_ex (the
 * output pointer is checked the same way, and a pixel response A is refused with WF_ERR_ARG because it
 * needs transformed copies of the inputs); the caller passes every input and the output buffer as before.
 *   - Scratch (the per-call coefficient tables) lives in one statically sized device array compiled into
 *     the library, 262,144 bytes, which every GPU that loads the library keeps until the process exits.
 *     Only H = W in {16, 32, 64, 128} fit; the larger sizes that wf_supported_size accepts (256, 512,
 *     1024) are rejected with WF_ERR_SHAPE before anything is launched.
 *   - The first call on each device looks up that array's device address (cudaGetSymbolAddress) with the
 *     device current; make that first call before any stream capture. Later calls reuse the address. The
 *     address belongs to the device's primary context: after cudaDeviceReset on a device, do not call
 *     this entry point on that device again in the same process.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.
 *   - All calls on a device share the one array and leave the last call's tables in it; every call
 *     rewrites what it reads before reading it, so nothing needs clearing, but calls that overlap on the
 *     GPU (other streams or host threads on the same device) race on it: serialise them.
 *   - The call waits for its own stream to finish before it returns, to read the status word.
 */
wf_status wf_sample_noalloc(const float* d, const float* Ndiag, const uint8_t* mask, const float* Pk, int32_t H,
                            int32_t W, uint64_t seed, const wf_sample_opts* opts, float* out, wf_stream_t stream);

/* ABI version of this header: (major << 16) | minor. */
int32_t wf_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WF_H_ */
