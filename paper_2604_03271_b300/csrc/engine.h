// engine.h -- host-side job engine behind the C ABI (internal).
//
// A request is one spectrum with its candidate range K = k_min..k_max; it owns
// one job per K.  Jobs live in a device job table (JobDev[SMC_MAX_SLOTS]);
// every kernel takes a device list of job-table slots and skips jobs that are
// not active, so one launch sequence advances every job of a batch by one
// tempering stage regardless of where each job is in its schedule.
#pragma once
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <array>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/smc.h"
#include "../../include/smc_kernels.h"
#include "kernels.h"
#include "prep.h"

namespace smc {

constexpr int MAX_SLOTS = 4096;
constexpr int LIST_AREA = 24 * MAX_SLOTS;  // ints of the device slot-list area
constexpr int CHUNK = 4;                   // stages per CUDA-graph launch
constexpr int NACTIVE_SLOTS = 64;
// internal status of setup_request: the context's memory budget or its job
// slots are taken for now (the serving loop retries later; the blocking entry
// points report SMC_ENOMEM)
constexpr int ST_NO_ROOM = 1000;

struct Tile {
    int J, G, R;  // R: register budget per thread (0: the tile's default)
};

struct Request {
    smc_job id = 0;
    int k_min = 0, k_max = 0, family = 0, bg = 0, bg_degree = 0, nbg = 0, p = 3;
    int n = 0;
    int noise = 0;                 // SMC_NOISE_*
    double noise_par[3] = {0, 0, 0};
    std::vector<double> ref_pos, ref_int;  // App. D reflections (all phases)
    std::vector<int32_t> ref_off;
    bool full = false;             // coupled-grid Metropolis kernel
    smc_options opts{};
    smc_priors pri{};
    std::vector<smc_prior> comp;
    std::vector<double> hx, hy, hs;  // host copies of the inputs
    const double *dx = nullptr, *dy = nullptr, *ds = nullptr;  // device inputs, if given
    bool fp64 = false;
    // device state
    void *spec_arena = nullptr;
    size_t spec_bytes = 0;
    SpecDev sd{};
    Tile tile{16, 1, 0};
    int n_pad = 0;
    std::vector<int> slots;
    std::vector<void *> job_arena;
    std::vector<size_t> job_bytes;
    // results
    // 0 queued, 1 running, 2 done.  Written by the serving thread or the
    // blocking entry points and read by smc_poll / smc_wait / smc_result under
    // another lock: atomic, and set to 2 only after every result field is
    // written (release), so that a reader that sees 2 sees the results
    std::atomic<int> state{0};
    int status = SMC_OK;
    int dim_max = 0;
    int64_t n_samples = 0;
    std::vector<double> log_z, p_k, mean, sdv;
    std::vector<int32_t> n_stages, job_status;
    int32_t selected_k = -1;      // argmax of log Z over successful jobs, ties to the lower K
    std::vector<float> samples;
    std::chrono::steady_clock::time_point t_submit, t_done;
    double latency_ms = 0.0;
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, used = 0;
    std::recursive_mutex mu;
    JobDev *d_jobs = nullptr;
    std::vector<JobDev> h_jobs;
    std::vector<int> free_slots;
    int *d_lists = nullptr;
    int *d_nactive = nullptr;
    int *h_nactive = nullptr;      // pinned, device-mapped, one entry per stage of a chunk
    int *h_nactive_dev = nullptr;  // its device alias
    // autotuned tiles: (family, n_max, J, G, R), under tmu (read when a
    // request is made, which submissions do without the engine lock)
    std::vector<std::array<int64_t, 5>> tiles;
    std::mutex tmu;
    // profiling (per-kernel events need the chunked graph: conditional bodies
    // take no event nodes)
    bool prof_events = false;
    int graph_mode = SMC_GRAPH_WHILE;  // smc_create_opts.graph_mode
    smc_profile prof{};
    std::map<smc_job, Request *> reqs;
    uint64_t next_id = 1;
    // serving
    std::thread worker;
    std::mutex qmu;
    std::condition_variable qcv, done_cv;
    std::deque<Request *> queue;
    std::vector<Request *> running;
    bool stop = false;
    bool worker_started = false;
};

// request construction and device resources
int make_request(Ctx &c, const smc_request &rq, bool on_device, Request *&out);
int setup_request(Ctx &c, Request &r, int64_t T_override = 0, int64_t S_override = 0);
void free_request_device(Ctx &c, Request &r);
size_t request_bytes(const Request &r);
Tile choose_tile(int family, int n);
int job_dim(int family, int K, int bg, int bg_degree);
int kernel_family(int family);

// run every job of the given requests to completion (batched FP32 path; plain
// FP64 requests run one job at a time) and collect their results
int run_requests(Ctx &c, std::vector<Request *> &reqs);
int finalize_requests(Ctx &c, std::vector<Request *> &reqs);
// `iters` stages of every active FP32 job of the requests (serving loop)
int run_chunk(Ctx &c, std::vector<Request *> &reqs, int iters);

// serving loop
void serve_loop(Ctx *c);

int cuda_status(cudaError_t e);

}  // namespace smc
