// pide2d_batch_*: many independent pricings on one GPU.
//
// Jobs are grouped by geometry (N, precision, departure order, number of
// steps).  Each group is split into chunks of at most `lanes` jobs.  A chunk
// gets one workspace lane per job and is advanced in lockstep by the
// multi-job time loop (solve_group in api.cu): one CUDA graph per chunk runs
// the whole time loop, every kernel of a theta step and of each fixed-point
// iteration launched once for the whole chunk, with the job in the grid's y
// (or z) dimension; jobs that have converged skip their blocks and the loops
// end on the device.  The precompute of each job (weights, rates, payoff)
// runs per job, from a few host threads.  Nothing here allocates device
// memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <map>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/pide2d.h"

namespace pide {
void set_global_error(const std::string& msg);
size_t group_scratch_bytes(int K, int n_steps);
pide2d_status solve_group(pide2d_t* const* hs, int K, void* scratch, int upb, std::string* err);
pide2d_status time_col_jobs(pide2d_t* const* hs, int K, void* scratch, int upb, int reps, double* ms, std::string* err);
int fft_units_per_block(int P, int prec_bytes);
void set_handle_stream(pide2d_t* h, void* stream);
}

namespace {

constexpr int kCreateThreads = 8;
constexpr int kTrialReps = 3;

// Launch shape of a geometry group, picked by timed trials on its first
// chunk (the column pass of the fixed-point iteration, the heaviest multi-job
// kernel): FFT units per block among 1x, 2x, 4x the single-job shape (up to
// 512 threads), then jobs per chunk among the chunk size and its half (a
// smaller chunk wins only if its time per job is 3% lower).
struct Shape {
    int upb = 0, lanes = 0;
    double us_per_job = 0.0;
};

pide2d_status tune_shape(pide2d_t* const* hs, int K, void* scratch, int N, int prec, Shape* out, std::string* err) {
    const int base = pide::fft_units_per_block(2 * N, prec == PIDE2D_FP64 ? 8 : 4);
    const int nt = (2 * N) / 16;
    Shape best;
    double best_ms = 1e300;
    int last = -1;
    for (int f : {1, 2, 4}) {
        const int u = std::min(base * f, std::max(1, 512 / nt));
        if (u == last) continue;
        last = u;
        double ms = 0.0;
        const pide2d_status st = pide::time_col_jobs(hs, K, scratch, u, kTrialReps, &ms, err);
        if (st != PIDE2D_OK) return st;
        if (ms < best_ms) {
            best_ms = ms;
            best.upb = u;
        }
    }
    best.lanes = K;
    best.us_per_job = 1e3 * best_ms / K;
    if (K / 2 >= 16) {
        double ms = 0.0;
        const pide2d_status st = pide::time_col_jobs(hs, K / 2, scratch, best.upb, kTrialReps, &ms, err);
        if (st != PIDE2D_OK) return st;
        const double per = 1e3 * ms / (K / 2);
        if (per < 0.97 * best.us_per_job) {
            best.lanes = K / 2;
            best.us_per_job = per;
        }
    }
    *out = best;
    return PIDE2D_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int job_steps(const pide2d_job& j);

// the longest time loop among the jobs (sizes the per-theta-step argument blobs)
int max_steps(const pide2d_job* jobs, int count) {
    int m = 1;
    for (int i = 0; i < count; ++i) m = std::max(m, job_steps(jobs[i]));
    return m;
}

pide2d_status lane_bytes(const pide2d_job* jobs, int count, size_t* out) {
    size_t mx = 0;
    for (int i = 0; i < count; ++i) {
        size_t b = 0;
        const pide2d_status s = pide2d_workspace_bytes(&jobs[i].grid, &b);
        if (s != PIDE2D_OK) return s;
        mx = std::max(mx, b);
    }
    *out = align256(mx);
    return PIDE2D_OK;
}

int job_steps(const pide2d_job& j) {
    return j.dt > 0.0 ? (int)std::llround(j.contract.maturity / j.dt) : 0;
}

}  // namespace

extern "C" {

pide2d_status pide2d_batch_workspace_bytes(const pide2d_job* jobs, int count, int lanes, size_t* bytes) {
    if (!jobs || count < 1 || lanes < 1 || lanes > 1024 || !bytes) {
        pide::set_global_error("pide2d_batch_workspace_bytes: invalid arguments");
        return PIDE2D_ERR_ARG;
    }
    size_t lb = 0;
    const pide2d_status s = lane_bytes(jobs, count, &lb);
    if (s != PIDE2D_OK) return s;
    const int L = std::min(lanes, count);
    *bytes = lb * (size_t)L + align256(pide::group_scratch_bytes(L, max_steps(jobs, count)));
    return PIDE2D_OK;
}

pide2d_status pide2d_batch_solve(const pide2d_job* jobs, int count, const pide2d_options* opts, int lanes,
                                 void* workspace, size_t workspace_bytes, double* prices, int* statuses,
                                 pide2d_batch_stats* stats) {
    if (!jobs || count < 1 || lanes < 1 || lanes > 1024 || !prices) {
        pide::set_global_error("pide2d_batch_solve: invalid arguments");
        return PIDE2D_ERR_ARG;
    }
    size_t lb = 0;
    pide2d_status s = lane_bytes(jobs, count, &lb);
    if (s != PIDE2D_OK) return s;
    lanes = std::min(lanes, count);
    const size_t need = lb * (size_t)lanes + align256(pide::group_scratch_bytes(lanes, max_steps(jobs, count)));
    if (!workspace || ((uintptr_t)workspace & 255) != 0 || workspace_bytes < need) {
        pide::set_global_error("pide2d_batch_solve: workspace too small or misaligned");
        return PIDE2D_ERR_WORKSPACE;
    }
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        pide::set_global_error("pide2d_batch_solve: no current CUDA device");
        return PIDE2D_ERR_CUDA;
    }
    char* ws = static_cast<char*>(workspace);
    void* scratch = ws + lb * (size_t)lanes;
    pide2d_options o{};
    if (opts) o = *opts;
    else o.kmax = 100, o.damping = 1;
    o.host_loop = 1;          // the handles never run a single-job device loop (the chunk graph does)

    // groups of one geometry, largest grids first
    std::map<std::tuple<int, int, int, int>, std::vector<int>, std::greater<std::tuple<int, int, int, int>>> groups;
    for (int j = 0; j < count; ++j) {
        const pide2d_grid& g = jobs[j].grid;
        const int order = g.sl_order == 0 ? 3 : g.sl_order;
        groups[std::make_tuple(g.n, g.precision, order, job_steps(jobs[j]))].push_back(j);
    }

    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
        pide::set_global_error("pide2d_batch_solve: cudaStreamCreate failed");
        return PIDE2D_ERR_CUDA;
    }
    std::vector<int> st(count, PIDE2D_OK);
    std::vector<pide2d_stats> js(count);
    std::string last_error;
    bool cuda_failed = false;
    pide2d_batch_stats bs{};
    const bool tune = !(opts && opts->fixed_shapes);

    for (auto& kv : groups) {
        const std::vector<int>& members = kv.second;
        Shape shape;                       // single-job shape, whole chunks, until the trials say otherwise
        bool tuned = false;
        for (size_t c0 = 0; c0 < members.size() && !cuda_failed; c0 += (size_t)lanes) {
            const int K = (int)std::min(members.size() - c0, (size_t)lanes);
            auto now = [] { return std::chrono::steady_clock::now(); };
            auto secs = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
                return std::chrono::duration<double>(b - a).count();
            };
            const auto tc0 = now();
            std::vector<pide2d_t*> hs(K, nullptr);
            // per-job precompute, a few handles at a time from host threads
            std::atomic<int> next(0);
            std::vector<std::string> errs(kCreateThreads);
            auto creator = [&](int tid) {
                cudaSetDevice(device);
                cudaStream_t cs = nullptr;
                if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
                    errs[tid] = "cudaStreamCreate failed";
                    return;
                }
                for (;;) {
                    const int q = next.fetch_add(1);
                    if (q >= K) break;
                    const int j = members[c0 + q];
                    const pide2d_job& job = jobs[j];
                    pide2d_t* h = nullptr;
                    const pide2d_status r = pide2d_create(&job.grid, &job.model, &job.contract, job.theta, job.dt,
                                                          job.fp_tol, &o, ws + lb * (size_t)q, lb, cs, &h);
                    if (r == PIDE2D_OK) {
                        pide::set_handle_stream(h, stream);     // create has finished on cs
                        hs[q] = h;
                    } else {
                        st[j] = r;
                        prices[j] = 0.0;
                        errs[tid] = pide2d_last_error(nullptr);
                    }
                }
                cudaStreamSynchronize(cs);
                cudaStreamDestroy(cs);
            };
            const int nt = std::min(kCreateThreads, K);
            std::vector<std::thread> pool;
            for (int t = 0; t < nt; ++t) pool.emplace_back(creator, t);
            for (auto& t : pool) t.join();
            for (const auto& e : errs)
                if (!e.empty()) last_error = e;
            // the created jobs run together
            std::vector<pide2d_t*> live;
            std::vector<int> live_idx;
            for (int q = 0; q < K; ++q)
                if (hs[q]) {
                    live.push_back(hs[q]);
                    live_idx.push_back(members[c0 + q]);
                }
            const auto tc1 = now();
            bs.create_s += secs(tc0, tc1);
            if (!live.empty() && tune && !tuned) {
                std::string err;
                const pide2d_status ts = tune_shape(live.data(), (int)live.size(), scratch, std::get<0>(kv.first),
                                                    std::get<1>(kv.first), &shape, &err);
                if (ts != PIDE2D_OK) {
                    for (int j : live_idx) st[j] = ts;
                    last_error = err;
                    cuda_failed = true;
                    live.clear();
                } else {
                    tuned = true;
                    if (bs.tuned < 8) {
                        bs.tune_n[bs.tuned] = std::get<0>(kv.first);
                        bs.tune_units[bs.tuned] = shape.upb;
                        bs.tune_lanes[bs.tuned] = shape.lanes;
                        bs.tune_us_per_job[bs.tuned] = shape.us_per_job;
                    }
                    bs.tuned += 1;
                }
            }
            const auto tl0 = now();
            bs.tune_s += secs(tc1, tl0);
            if (!live.empty()) {
                std::string err;
                pide2d_status gs = PIDE2D_OK;
                const int sub = shape.lanes > 0 ? shape.lanes : (int)live.size();
                for (size_t q0 = 0; q0 < live.size() && gs == PIDE2D_OK; q0 += (size_t)sub) {
                    const int Kq = (int)std::min(live.size() - q0, (size_t)sub);
                    gs = pide::solve_group(live.data() + q0, Kq, scratch, shape.upb, &err);
                }
                if (gs != PIDE2D_OK) {
                    for (int j : live_idx) st[j] = gs;
                    last_error = err;
                    if (gs == PIDE2D_ERR_CUDA) cuda_failed = true;
                } else {
                    for (size_t q = 0; q < live.size(); ++q) {
                        const int j = live_idx[q];
                        const pide2d_status r = pide2d_solve(live[q], &prices[j], nullptr, &js[j]);
                        st[j] = r;
                        if (r != PIDE2D_OK) last_error = pide2d_last_error(live[q]);
                    }
                }
            }
            bs.loop_s += secs(tl0, now());
            for (auto* h : hs)
                if (h) pide2d_destroy(h);
        }
    }
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);

    pide2d_status worst = PIDE2D_OK;
    for (int j = 0; j < count; ++j) {
        if (cuda_failed && st[j] == PIDE2D_OK && js[j].steps_done == 0) st[j] = PIDE2D_ERR_CUDA;
        if (statuses) statuses[j] = st[j];
        if (st[j] == PIDE2D_OK || st[j] == PIDE2D_ERR_NOT_CONVERGED) {
            bs.jobs_done += 1;
            bs.fp_iters_total += js[j].fp_iters_total;
            bs.cell_iters += js[j].cell_iters;
        }
        if (st[j] != PIDE2D_OK) {
            bs.failures += 1;
            if (worst == PIDE2D_OK || st[j] == PIDE2D_ERR_CUDA) worst = (pide2d_status)st[j];
        }
    }
    if (stats) *stats = bs;
    if (!last_error.empty()) pide::set_global_error(last_error);
    return worst;
}

}  // extern "C"
