// kernels.h -- host-side launchers of the sampler's kernels (internal).
// Every launcher takes a device array `slots` of job-table indices; kernels
// skip jobs that are not active.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "smc_device.cuh"

namespace smc {

// Philox words for n counters (testing / profiling).
cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t n,
                          cudaStream_t s);

// Prior draws at beta = 0 for the listed jobs (all T particles of each), FP64
// draws stored as FP32 (fast jobs) or FP64 (plain jobs).
cudaError_t launch_prior_init(JobDev *jobs, const int *slots, int nslots, int max_T,
                              cudaStream_t s);

// Energies of all T particles of each listed job (FP32 jobs: warp per particle,
// Kahan-compensated; FP64 jobs: thread per particle).
cudaError_t launch_energy(JobDev *jobs, const int *slots, int nslots, int max_T, bool fp64,
                          cudaStream_t s);

// Tempering step of every active listed job: ESS bisection, log Z increment,
// step sizes, quantised weights.  Tempering step of every job in slots (FP64 jobs: one cluster kernel; FP32
// jobs: search, weights and finish kernels).  t_max: largest T of the jobs.
constexpr int RW_SPLIT_MAX = 64;
int rw_split(int64_t T);  // CTAs per FP32 job in the weights kernel
cudaError_t launch_reweight(JobDev *jobs, const int *slots, int nslots, bool fp64, int64_t t_max,
                            cudaStream_t s);
cudaError_t launch_temper32(JobDev *jobs, const int *slots, int nslots, int64_t t_max, cudaStream_t s);

// Systematic resampling of given integer weights (one CTA).
cudaError_t launch_resample_raw(const unsigned long long *q, int T, int M, uint32_t u32, int *anc,
                                cudaStream_t s);

// Systematic resampling (one CTA per job) and the particle copy.
cudaError_t launch_resample(JobDev *jobs, const int *slots, int nslots, cudaStream_t s);
cudaError_t launch_gather(JobDev *jobs, const int *slots, int nslots, int64_t max_elems,
                          bool fp64, cudaStream_t s);

// Fused FP32 Metropolis stage of one bucket (family, points per lane J, warps
// per chain G, all listed jobs sharing them); grid 0 = one wave of resident CTAs.
// family = FAM_* of the peaks, | MH_COUPLED for the coupled-grid kernel (Shirley
// background and/or model variance).
constexpr int MH_COUPLED = 16;
// kcap: most peaks (phases) of the launch's jobs; the phase kernel then gets
// dynamic shared memory for that many cached profiles per chain (if it fits)
// R: register budget per thread of the fused kernel (0: the tile's default;
// 64, 80, 96 or 128 for four- and eight-warp chains with J = 4, 8, 16)
cudaError_t launch_mh(JobDev *jobs, const int *slots, int nslots, int family, int J, int G, int R,
                      int grid, cudaStream_t s, int kcap = 0);
bool mh_tile_supported(int family, int J, int G, int R = 0);
int mh_resident_grid(int family, int J, int G, int R = 0, int kcap = 0);

// Plain FP64 Metropolis stage (thread per chain, full energy per proposal).
cudaError_t launch_mh_plain(JobDev *jobs, const int *slots, int nslots, int max_S,
                            cudaStream_t s);

// Advance stage counters, retire finished jobs, count the jobs still active
// into *n_active (device) and *n_active_host (host-mapped, may be NULL).
cudaError_t launch_stage_end(JobDev *jobs, const int *slots, int nslots, int *n_active,
                             int *n_active_host, cudaStream_t s);

// Same, as the last node of a whole-run graph: sets the while-node condition
// (any job active and fewer than max_iter stages run, counted in *iter).
cudaError_t launch_stage_end_cond(JobDev *jobs, const int *slots, int nslots, int *n_active,
                                  cudaGraphConditionalHandle cond, int *iter, int max_iter,
                                  cudaStream_t s);

// Posterior summaries (peaks sorted by centre) and natural-value samples;
// row a of mean/sd/samples belongs to slots[a].  Every job has T particles and
// at most d_max components / k_max peaks.  part: nslots * finalize_split(T) *
// 2 * dim_stride doubles of scratch; counters: nslots ints, zero on entry
// (left zero on exit).
int finalize_split(int64_t T);
cudaError_t launch_finalize(JobDev *jobs, const int *slots, int nslots, int d_max, int k_max, int64_t T,
                            double *mean, double *sd, float *samples, int dim_stride,
                            int64_t sample_stride, double *part, int *counters, cudaStream_t s);

}  // namespace smc
