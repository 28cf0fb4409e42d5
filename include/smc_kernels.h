/*
 * smc_kernels.h -- step-level entry points of the sampler, for parity testing
 * and profiling of each kernel on its own.  They run exactly the kernels that
 * smc_run launches, on a temporary one-job set, and copy results back.
 *
 * All array arguments are HOST arrays (copied in and out by the call).
 * Particles are passed as natural parameter values, row-major [count][d],
 * components in the order documented in smc.h.  `precision` selects the
 * kernel family: 0 = the FP32-energy batched kernels, 1 = the plain FP64 ones.
 * A request is validated as smc_run validates it, with energy_fp64 taken from
 * `precision` (so a request that smc_run rejects in FP32 -- Poisson counts on
 * Gaussian peaks without a background -- is rejected here at precision 0).
 * Every call returns an SMC_* status and leaves outputs untouched on error.
 */
#ifndef SMC_KERNELS_H
#define SMC_KERNELS_H

#include "smc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 (Salmon et al., SC'11) evaluated on the device:
 * out[4i..4i+3] = Philox(ctr[4i..4i+3], key = (seed lo, seed hi)), i < n. */
int smc_k_philox(smc_ctx *ctx, uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n);

/* Energy E = 1/2 sum ((y - f)/sigma)^2 of `count` particles for the model of
 * spec with K peaks (forward model Eq. (1); Gaussian likelihood, App. C Eq. (C2)).
 * spec->priors fixes each component's sampling coordinate. */
int smc_k_energy(smc_ctx *ctx, const smc_request *spec, int32_t K, const double *nat,
                 int64_t count, int32_t precision, double *E_out);

/* Prior draws at beta = 0 (Eq. (9)) for particles 0..count-1 with spec->opts->seed:
 * natural values [count][d] and their energies. */
int smc_k_prior(smc_ctx *ctx, const smc_request *spec, int32_t K, int64_t count,
                int32_t precision, double *nat_out, double *E_out);

/* Tempering step for energies E[T] at inverse temperature beta: the increment
 * delta from the ESS bisection (ESS >= rho T), the log-evidence increment
 * log mean exp(-delta E) (Eq. (11)), whether the step reached beta = 1, and the
 * integer-quantised weights q[T] = floor(exp(-delta (E - min E)) 2^40) used by
 * the resampler (q_out may be NULL).  precision 0 rounds E to FP32 first. */
int smc_k_reweight(smc_ctx *ctx, const double *E, int64_t T, double beta, double rho,
                   int32_t precision, double *delta, double *logz_inc, int32_t *final_step,
                   uint64_t *q_out);

/* Allocation-free variant of smc_k_reweight, for callers that cannot
 * allocate device memory (a host framework that owns every allocation, or a
 * service that must not grow device memory once running).  No counterpart in
 * the paper: same kernel and results as smc_k_reweight, but the caller passes
 * DEVICE arrays -- E_dev (T floats if precision is 0, T doubles if 1) and
 * q_dev (T uint64 outputs) -- and the kernel's scratch (its job descriptor and
 * FP64 weights) is a fixed static device array of this library, sized for at
 * most SMC_STATIC_MAX_PARTICLES particles (about 8 MiB, held by every GPU that
 * loads the library until exit).  Runs on the current device and cuda_stream
 * (NULL = default stream) and returns after the stream has finished the step.
 * T above the maximum returns SMC_EINVAL.  Each call outside a stream capture
 * looks up the scratch address (cudaGetSymbolAddress) on the current device,
 * so calls stay valid after a device reset; a call inside a capture reuses the
 * last address found on that device, so make one call on each device before
 * any capture.  Calls share the scratch: calls that overlap on the GPU race. */
#define SMC_STATIC_MAX_PARTICLES (1 << 20)
int smc_k_reweight_static(const void *E_dev, int64_t T, double beta, double rho,
                          int32_t precision, uint64_t *q_dev, double *delta, double *logz_inc,
                          int32_t *final_step, void *cuda_stream);

/* Systematic resampling of M ancestors from integer weights q[T] with the
 * uniform word u32: a_m = min{i : C_i > floor((m Q + floor(u32 Q / 2^32)) / M)},
 * C the inclusive prefix sum of q, Q = C_{T-1}. */
int smc_k_resample(smc_ctx *ctx, const uint64_t *q, int64_t T, int64_t M, uint32_t u32,
                   int32_t *anc);

/* One Metropolis stage (Sec. II B 4) on S chain starts at inverse temperature
 * beta and stage counter `stage`, with step sizes step[d] in sampling
 * coordinates and spec->opts->sweeps sweeps.  Outputs the chains' final (or,
 * if waste_free, every sweep's) states and energies, and per-component accept
 * and proposal counts acc[d], prop[d]. */
int smc_k_mh_stage(smc_ctx *ctx, const smc_request *spec, int32_t K, const double *nat_start,
                   const double *E_start, int64_t S, const double *step, double beta,
                   uint32_t stage, int32_t precision, double *nat_out, double *E_out,
                   int64_t *acc, int64_t *prop);

/* Tile of the fused Metropolis kernel for FP32 jobs of `family` whose grid
 * has at most n_max points: J points per lane (4, 8, 12, 16; also 24, 32 for
 * Gaussian/Lorentzian) and G warps per chain (1, 2, 4, 8; 16 with J <= 8),
 * 32 G J >= N, and the register budget per thread `regs`: 0 for the tile's
 * default, or 64, 80, 96, 128 for G = 4 or 8 with J = 4, 8, 16 (fewer
 * registers, more resident warps).  family | SMC_TILE_COUPLED sets the tile of
 * the coupled-grid kernel (Shirley background or model variance: J = 4 or 8,
 * regs 0); SMC_XRD_PHASE (always coupled) that of the phase kernel (J = 4 or
 * 8, regs 0).  Entries are matched in the order they were set; the first
 * whose family matches and n_max >= N wins; without a match a
 * padding-minimising default is used.  J = 0 clears the table.  SMC_EINVAL
 * for a tile that is not compiled.  Used by the autotuner. */
#define SMC_TILE_COUPLED 16
int smc_set_tile(smc_ctx *ctx, int32_t family, int64_t n_max, int32_t J, int32_t G, int32_t regs);

/* Profiling counters of a context, accumulated over the runs finished since
 * the last smc_profile_reset.  Kernel classes: 0 reweight (tempering step),
 * 1 resample, 2 gather (particle copy), 3 Metropolis, 4 stage end.  With
 * events enabled, every batched stage records CUDA events around each kernel
 * class on the context's stream (inside the CUDA graph); `launches` counts
 * kernel launches of stages in which at least one job was active and `ms` the
 * summed event time of those launches.  The algorithmic counters are exact
 * counts made by the kernels themselves:
 *   point_evals  grid-point evaluations of evaluated proposals (plus the
 *                prior-draw energies), the "particle-point evaluations";
 *   sfu_ops      SFU operations (EX2, RCP) the centre/width proposals need:
 *                N per Gaussian or Lorentzian evaluation, 2 N per pseudo-Voigt;
 *   ex2_ops / rcp_ops  the same split by operation (Gaussian: EX2,
 *                Lorentzian: RCP, pseudo-Voigt: one of each per point), plus,
 *                with the model variance, one RCP and one LG2 (lg2_ops) per
 *                point of every evaluated proposal (not part of sfu_ops);
 *   gather_bytes bytes the particle copy must move (read + write), per stage;
 *   resample_bytes bytes the resampler must move (q read, ancestors written);
 *   h2d_bytes / d2h_bytes  host<->device bytes the calls copied;
 *   max_batch_requests  the most requests (spectra) whose jobs advanced in
 *                the same launches: > 1 shows that batched or served
 *                requests shared kernels on the device;
 *   peak_point_evals  grid-point evaluations of evaluated peak-component
 *                proposals in the fused peak kernel (Gaussian, Lorentzian,
 *                pseudo-Voigt peaks with a Chebyshev background), each costing
 *                peak_sfu_per_eval SFU operations in the method's own count
 *                (one new peak evaluation per unit: EX2 for a Gaussian, RCP for
 *                a Lorentzian, both for a pseudo-Voigt; of the last job read). */
typedef struct {
    int64_t launches[5];
    double ms[5];
    double point_evals, sfu_ops, gather_bytes, resample_bytes;
    double h2d_bytes, d2h_bytes;
    int64_t stages, jobs;
    double ex2_ops, rcp_ops, lg2_ops;
    int64_t max_batch_requests;
    double peak_point_evals, peak_sfu_per_eval;
} smc_profile;

int smc_profile_reset(smc_ctx *ctx, int32_t enable_events);
int smc_profile_read(smc_ctx *ctx, smc_profile *out);

/* Measured throughput of one SFU (MUFU) operation on the current device:
 * op 0 = EX2 (ex2.approx.ftz.f32), op 1 = RCP (rcp.approx.ftz.f32), the two
 * transcendentals of the peak shapes, op 2 = LG2 (lg2.approx.ftz.f32, the
 * model variance's logarithm).  Runs a dependency-free stream of the
 * operation on every SM (twelve launches, about 0.25 s, on cuda_stream; the
 * best of the last four counts) and returns results per second over the whole
 * device, the SM clock the blocks saw (clock64 cycles over globaltimer
 * nanoseconds, MHz) and results per clock per SM at that clock.  The paper
 * has no counterpart: it is the denominator of the Metropolis kernel's
 * roofline.  Allocates and frees its own small buffers. */
int smc_k_mufu_rate(int32_t op, double *ops_per_s, double *lanes_per_clk_sm, double *sm_mhz,
                    void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SMC_KERNELS_H */
