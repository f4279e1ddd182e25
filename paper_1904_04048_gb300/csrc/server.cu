// Serving loop: continuous batching of independent simulations.
//
// Requests (grid, scheme, Courant number, step count, initial data) arrive at
// any time from any thread.  A scheduler thread owns the GPU work: each round
// it admits queued requests in arrival order while the device-memory budget
// and the slot limit allow, runs the first step (Eq. A1) of the newly
// admitted ones in one batched launch, advances every resident simulation by
// up to `quantum` two-steps (Eq. A2) in one batched run (one launch per
// sub-quantum over the tiles of all of them), and retires the simulations
// that reached their step count: FP64 norms copied to the host, the final
// level copied out if requested, completion time stamped, memory released.
// Requests admitted while others are running join them at the next round, so
// their work overlaps on the device.  Every simulation is stepped by the same
// per-node arithmetic as a single handle, so a result does not depend on what
// else was resident.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "wave2d_impl.cuh"

namespace w2d {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// u0 = amp exp(-|x - c|^2 / (2 sigma^2)), v0 = 0 on the zero-boundary node set
// x = (i + 1) h.
__global__ void k_gaussian_ic(double* u0, double* v0, int nx, int ny, double h, double amp, double cx, double cy,
                              double sigma) {
    const long long n = (long long)nx * ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % nx), j = (int)(q / nx);
        const double dx = (i + 1) * h - cx, dy = (j + 1) * h - cy;
        u0[q] = amp * exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma));
        v0[q] = 0.0;
    }
}

struct Pending {
    wave2d_request r;
    std::vector<double> u0, v0;  // host copies when the request brought arrays
    double t_submit = 0;
};

struct Active {
    Pending p;
    wave2d_t h = nullptr;
    int64_t remaining = 0;
    int64_t bytes = 0;
    double t_admit = 0;
    int failed = WAVE2D_OK;  // status of a step that failed for this request (it is retired with it)
    uint64_t id = 0;         // admission number: identifies the simulation (a handle's address may recur)
};

}  // namespace
}  // namespace w2d

using namespace w2d;

struct wave2d_server {
    int64_t budget = 0;
    int max_resident = 0;
    int quantum = 64;
    int kernel = WAVE2D_KERNEL_STREAM;  // batched runs: register streaming (the zero boundary of every request)
    int Tq = 4, OH = 64;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Pending> queue;
    std::deque<wave2d_completion> done;
    std::vector<Active> resident;
    int64_t used = 0;
    int64_t submitted = 0, completed = 0;
    int64_t node_updates = 0;
    int64_t rounds = 0;
    int max_resident_seen = 0;
    bool stop = false;
    int fatal = 0;
    std::string fatal_msg;
    std::thread worker;
    // pipeline (scheduler thread only): the batch that advances the resident
    // set, requests whose norms are on their way to the host, and the rounds
    // still executing (bounded, and timed for the busy fraction)
    wave2d_batch_t batch = nullptr;
    std::vector<uint64_t> batch_members;  // admission numbers of the batch's members, in order
    uint64_t next_id = 1;
    int batch_rows = 0;     // strip rows of the batch's current plan
    bool auto_rows = true;  // strip rows chosen per round (false: fixed by opt->tile_h)
    int num_sms = 0;
    struct Retiring {
        std::vector<Active> items;
        double* norms = nullptr;  // pinned, two per item
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
    };
    std::deque<Retiring> retiring;
    std::vector<std::pair<double*, size_t>> pinned_pool;
    struct Mark {
        cudaEvent_t start = nullptr, end = nullptr;
    };
    std::deque<Mark> marks;
    double busy_s = 0;
};

namespace {

int64_t required_bytes_of(int nx, int ny, int dtype) {
    const int64_t pitch = (int64_t)round_up((size_t)nx + 2 * kGhost, 32);
    const int64_t rows = ny + 2 * kGhost;
    const int64_t elem = dtype == WAVE2D_F64 ? 8 : 4;
    const int64_t plane = (int64_t)round_up((size_t)(pitch * rows * elem), 1024);
    const int nplanes = dtype == WAVE2D_F32 ? 4 : (dtype == WAVE2D_F32X2 ? 4 : 2);
    const int64_t blocks = std::max<int64_t>((int64_t)((nx + 31) / 32) * ((ny + 7) / 8), 64 * 1024);
    const int64_t scratch = (int64_t)round_up(blocks * 32, 256) + 1024 + 2 * (int64_t)round_up((2 * (size_t)nx + 2 * ny) * 8, 256);
    return nplanes * plane + scratch;
}

void fail_round(wave2d_server* s, int rc) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->fatal) {
        s->fatal = rc;
        s->fatal_msg = wave2d_last_error();
    }
}

void complete(wave2d_server* s, Active& a, int status, double l2, double linf, int64_t k) {
    wave2d_completion c{};
    c.tag = a.p.r.tag;
    c.status = status;
    c.l2 = l2;
    c.linf = linf;
    c.k = k;
    c.t_submit = a.p.t_submit;
    c.t_admit = a.t_admit;
    c.t_done = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(c);
    s->completed += 1;
    s->used -= a.bytes;
    s->done_cv.notify_all();
}

double* pinned_get(wave2d_server* s, size_t n, size_t& cap) {
    for (size_t i = 0; i < s->pinned_pool.size(); ++i)
        if (s->pinned_pool[i].second >= n) {
            auto pr = s->pinned_pool[i];
            s->pinned_pool.erase(s->pinned_pool.begin() + i);
            cap = pr.second;
            return pr.first;
        }
    double* p = nullptr;
    cap = std::max<size_t>(n, 64);
    if (cudaMallocHost(&p, cap * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Collect finished work: rounds whose end mark has passed (their GPU time),
// and retirements whose norms have arrived (their completions).  block:
// wait for the oldest round or retirement first.
void reap(wave2d_server* s, bool block) {
    if (block) {
        if (!s->retiring.empty()) cudaEventSynchronize(s->retiring.front().ev);
        else if (!s->marks.empty()) cudaEventSynchronize(s->marks.front().end);
    }
    while (!s->marks.empty()) {
        auto& m = s->marks.front();
        const cudaError_t q = cudaEventQuery(m.end);
        if (q == cudaErrorNotReady) break;
        float ms = 0;
        if (q == cudaSuccess && cudaEventElapsedTime(&ms, m.start, m.end) == cudaSuccess) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->busy_s += ms * 1e-3;
        }
        cudaGetLastError();
        cudaEventDestroy(m.start);
        cudaEventDestroy(m.end);
        s->marks.pop_front();
    }
    while (!s->retiring.empty()) {
        auto& r = s->retiring.front();
        const cudaError_t q = cudaEventQuery(r.ev);
        if (q == cudaErrorNotReady) break;
        int rc = WAVE2D_OK;
        if (q != cudaSuccess) {
            rc = cuda_fail(q, "batched norms");
            fail_round(s, rc);
        }
        for (size_t i = 0; i < r.items.size(); ++i) {
            Active& a = r.items[i];
            double l2 = NAN, linf = NAN;
            int st = rc;
            if (rc == WAVE2D_OK) {
                l2 = r.norms[2 * i];
                linf = r.norms[2 * i + 1];
                if (!std::isfinite(l2) || !std::isfinite(linf)) st = WAVE2D_ERR_NONFINITE;
            }
            complete(s, a, st, l2, linf, a.p.r.steps + 1);
        }
        if (r.norms) s->pinned_pool.push_back({r.norms, r.cap});
        cudaEventDestroy(r.ev);
        s->retiring.pop_front();
    }
}

// One scheduling round; returns false when there is nothing to do.  The host
// queues a round's work (first steps of the admitted requests, one quantum of
// every resident simulation, the norms of those that finish) without waiting
// for the GPU, and runs at most two rounds ahead of it.
bool round_once(wave2d_server* s) {
    reap(s, false);
    while (s->marks.size() >= 2) reap(s, true);

    // 1. admission (FIFO, budget and slots)
    std::vector<Active> admitted;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (!s->queue.empty() && (int)(s->resident.size() + admitted.size()) < s->max_resident) {
            Pending& p = s->queue.front();
            const int64_t need = required_bytes_of(p.r.nx, p.r.ny, WAVE2D_F32);
            if (s->used + need > s->budget && !(s->resident.empty() && admitted.empty() && s->used == 0)) break;
            Active a;
            a.p = std::move(p);
            a.bytes = need;
            a.t_admit = now_s();
            a.remaining = a.p.r.steps;
            a.id = s->next_id++;
            s->used += need;
            admitted.push_back(std::move(a));
            s->queue.pop_front();
        }
    }
    if (admitted.empty() && s->resident.empty()) {
        if (s->retiring.empty() && s->marks.empty()) return false;
        reap(s, true);
        return true;
    }
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    if (cudaEventCreate(&ev_start) == cudaSuccess) cudaEventRecord(ev_start, s->stream);

    // 2. create handles and run the first step of the admitted requests
    if (!admitted.empty()) {
        std::vector<wave2d_t> hs_host, hs_pulse;
        std::vector<const double*> u_host, v_host;
        std::vector<Active*> pulses;
        std::vector<Active> ok_list;
        for (Active& a : admitted) {
            wave2d_grid g{};
            g.nx = a.p.r.nx;
            g.ny = a.p.r.ny;
            g.bc = WAVE2D_BC_ZERO;
            g.dtype = WAVE2D_F32;
            g.flags = a.p.r.flags;
            g.stream = s->stream;
            int rc = wave2d_create(&g, a.p.r.h, a.p.r.tau, a.p.r.c, a.p.r.scheme, &a.h);
            if (rc != WAVE2D_OK) {
                complete(s, a, rc, NAN, NAN, 0);
                continue;
            }
            ok_list.push_back(std::move(a));
        }
        admitted.swap(ok_list);
        for (Active& a : admitted) {
            if (!a.p.u0.empty()) {
                hs_host.push_back(a.h);
                u_host.push_back(a.p.u0.data());
                v_host.push_back(a.p.v0.data());
            } else {
                hs_pulse.push_back(a.h);
                pulses.push_back(&a);
            }
        }
        wave2d_tune opt{};
        opt.use_graph = 0;
        if (!hs_host.empty()) {
            wave2d_batch_t b = nullptr;
            int rc = wave2d_batch_create(hs_host.data(), (int)hs_host.size(), &opt, &b);
            if (rc == WAVE2D_OK) rc = wave2d_batch_first_step(b, u_host.data(), v_host.data(), 0);
            wave2d_batch_destroy(b);
            if (rc != WAVE2D_OK) {
                for (Active& a : admitted)
                    if (!a.p.u0.empty()) a.failed = rc;
                fail_round(s, rc);
            }
        }
        if (!hs_pulse.empty()) {
            size_t total = 0;
            for (Active* a : pulses) total += 2 * (size_t)a->p.r.nx * a->p.r.ny;
            Allocator al = current_allocator();
            double* stage = (double*)dev_alloc(al, total * sizeof(double), s->stream);
            if (!stage) {
                // the requests of this round fail; the server keeps serving
                const int rc = set_error(WAVE2D_ERR_OOM, "initial-data staging allocation failed");
                for (Active* a : pulses) a->failed = rc;
            } else {
                std::vector<const double*> pu, pv;
                double* p = stage;
                for (Active* a : pulses) {
                    const size_t nn = (size_t)a->p.r.nx * a->p.r.ny;
                    k_gaussian_ic<<<(int)std::min<size_t>((nn + 255) / 256, 4096), 256, 0, s->stream>>>(
                        p, p + nn, a->p.r.nx, a->p.r.ny, a->p.r.h, a->p.r.pulse_amp, a->p.r.pulse_cx,
                        a->p.r.pulse_cy, a->p.r.pulse_sigma);
                    g_launches.fetch_add(1);
                    pu.push_back(p);
                    pv.push_back(p + nn);
                    p += 2 * nn;
                }
                wave2d_batch_t b = nullptr;
                int rc = wave2d_batch_create(hs_pulse.data(), (int)hs_pulse.size(), &opt, &b);
                if (rc == WAVE2D_OK) rc = wave2d_batch_first_step(b, pu.data(), pv.data(), 1);
                wave2d_batch_destroy(b);
                dev_free(al, stage, total * sizeof(double), s->stream);  // in stream order, after the first step
                if (rc != WAVE2D_OK) {
                    for (Active* a : pulses) a->failed = rc;
                    fail_round(s, rc);
                }
            }
        }
        int64_t first_nodes = 0;
        for (Active& a : admitted) {
            if (a.failed == WAVE2D_OK) first_nodes += (int64_t)a.p.r.nx * a.p.r.ny;
            s->resident.push_back(std::move(a));
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->node_updates += first_nodes;  // the first level of each request
        s->max_resident_seen = std::max<int>(s->max_resident_seen, (int)s->resident.size());
    }

    // 3. advance every resident simulation (not failed) by up to one quantum,
    //    with the batch kept from round to round while its members stay
    std::vector<wave2d_t> hs;
    std::vector<uint64_t> ids;
    std::vector<int64_t> steps(s->resident.size(), 0), run_steps;
    int64_t nodes = 0;
    for (size_t i = 0; i < s->resident.size(); ++i) {
        Active& a = s->resident[i];
        if (a.failed != WAVE2D_OK) continue;
        steps[i] = std::min<int64_t>(a.remaining, s->quantum);
        hs.push_back(a.h);
        ids.push_back(a.id);
        run_steps.push_back(steps[i]);
        nodes += (int64_t)a.p.r.nx * a.p.r.ny * steps[i];
    }
    if (!hs.empty()) {
        int rc = WAVE2D_OK;
        // Register streaming: the tallest strips (64, 32 or 16 rows) that still
        // give a full wave of warps over the resident set; few resident
        // simulations make short launches, which keep the round (and so the
        // latency of every request in it) short.
        int rows = s->OH;
        if (s->kernel == WAVE2D_KERNEL_STREAM && s->auto_rows) {
            const int wave = 16 * std::max(1, s->num_sms);
            rows = 16;
            for (int L : {64, 32}) {
                int64_t strips = 0;
                for (wave2d_t h : hs) strips += (int64_t)((h->nx + 111) / 112) * ((h->ny + L - 1) / L);
                if (strips >= wave) {
                    rows = L;
                    break;
                }
            }
        }
        if (!s->batch) {
            wave2d_tune opt{};
            opt.use_graph = 0;
            opt.kernel = s->kernel;
            opt.temporal_t = s->Tq;
            opt.tile_h = rows;
            rc = wave2d_batch_create(hs.data(), (int)hs.size(), &opt, &s->batch);
            if (rc == WAVE2D_OK) s->batch_members = ids;
            s->batch_rows = rows;
        } else if (ids != s->batch_members || rows != s->batch_rows) {
            rc = batch_set_handles(s->batch, hs.data(), (int)hs.size(), rows);
            if (rc == WAVE2D_OK) s->batch_members = ids;
            s->batch_rows = rows;
        }
        if (rc == WAVE2D_OK) rc = wave2d_batch_run(s->batch, run_steps.data());
        if (rc != WAVE2D_OK) {
            // every simulation of the failed run is retired with its status;
            // none of its levels count as done
            for (Active& a : s->resident)
                if (a.failed == WAVE2D_OK) a.failed = rc;
            nodes = 0;
            fail_round(s, rc);
        }
    }

    // 4. retire finished and failed simulations: the norms of those that
    //    finished in one launch, copied to pinned memory and collected when
    //    the copy's event has passed; handles released in stream order
    std::vector<Active> still, finishing;
    for (size_t i = 0; i < s->resident.size(); ++i) {
        Active& a = s->resident[i];
        if (a.failed != WAVE2D_OK) {
            release_handle_nosync(a.h);
            a.h = nullptr;
            complete(s, a, a.failed, NAN, NAN, 0);
            continue;
        }
        a.remaining -= steps[i];
        if (a.remaining > 0) still.push_back(std::move(a));
        else finishing.push_back(std::move(a));
    }
    s->resident.swap(still);
    if (!finishing.empty()) {
        wave2d_server::Retiring r;
        std::vector<wave2d*> fh;
        for (Active& a : finishing) fh.push_back(a.h);
        r.norms = pinned_get(s, 2 * finishing.size(), r.cap);
        int rc = r.norms ? batch_norms_async(fh.data(), (int)fh.size(), s->stream, current_allocator(), r.norms)
                         : set_error(WAVE2D_ERR_OOM, "pinned norm buffer allocation failed");
        if (rc == WAVE2D_OK && cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess)
            rc = set_error(WAVE2D_ERR_CUDA, "event create failed");
        for (Active& a : finishing) {
            if (rc == WAVE2D_OK && a.p.r.out_field)
                wave2d_get_state(a.h, nullptr, a.p.r.out_field, nullptr);  // synchronises: only when asked
            release_handle_nosync(a.h);
            a.h = nullptr;
        }
        if (rc == WAVE2D_OK) {
            cudaEventRecord(r.ev, s->stream);
            r.items = std::move(finishing);
            s->retiring.push_back(std::move(r));
        } else {
            if (r.norms) s->pinned_pool.push_back({r.norms, r.cap});
            for (Active& a : finishing) complete(s, a, rc, NAN, NAN, 0);
        }
    }
    if (ev_start && cudaEventCreate(&ev_end) == cudaSuccess) {
        cudaEventRecord(ev_end, s->stream);
        s->marks.push_back({ev_start, ev_end});
    } else if (ev_start) {
        cudaEventDestroy(ev_start);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->node_updates += nodes;
        s->rounds += 1;
    }
    return true;
}

void worker_main(wave2d_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool idle = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const bool empty = s->queue.empty() && s->resident.empty();
            if (s->stop && empty && s->retiring.empty() && s->marks.empty()) break;
            if (empty && s->retiring.empty() && s->marks.empty()) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            idle = empty;
        }
        if (idle) reap(s, true);  // only results in flight: collect them
        else round_once(s);
    }
    if (s->batch) {
        wave2d_batch_destroy(s->batch);
        s->batch = nullptr;
    }
    cudaStreamSynchronize(s->stream);
    for (auto& pr : s->pinned_pool) cudaFreeHost(pr.first);
    s->pinned_pool.clear();
}

}  // namespace

extern "C" {

int64_t wave2d_required_bytes(int nx, int ny, int dtype) {
    if (nx < 1 || ny < 1 || (dtype != WAVE2D_F64 && dtype != WAVE2D_F32 && dtype != WAVE2D_F32X2))
        return set_error(WAVE2D_ERR_ARG, "bad grid");
    return required_bytes_of(nx, ny, dtype);
}

int wave2d_server_create(int64_t budget_bytes, int max_resident, int quantum, const wave2d_tune* opt, void* stream,
                         wave2d_server_t* out) {
    if (!out || budget_bytes <= 0 || max_resident < 1 || quantum < 1)
        return set_error(WAVE2D_ERR_ARG, "server needs a positive budget, slot count and quantum");
    *out = nullptr;
    wave2d_server* s = new (std::nothrow) wave2d_server();
    if (!s) return set_error(WAVE2D_ERR_OOM, "host allocation failed");
    s->budget = budget_bytes;
    s->max_resident = max_resident;
    s->quantum = quantum;
    if (opt && opt->kernel == WAVE2D_KERNEL_TEMPORAL) {
        s->kernel = WAVE2D_KERNEL_TEMPORAL;
        s->OH = 32;
    }
    if (opt && opt->temporal_t >= 1 && opt->temporal_t <= 4) s->Tq = opt->temporal_t;
    if (opt && s->kernel == WAVE2D_KERNEL_TEMPORAL && (opt->tile_h == 32 || opt->tile_h == 64)) s->OH = opt->tile_h;
    if (opt && s->kernel == WAVE2D_KERNEL_STREAM && opt->tile_h >= 8 && opt->tile_h <= 1024) {
        s->OH = opt->tile_h;
        s->auto_rows = false;
    }
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    s->stream = (cudaStream_t)stream;
    if (e == cudaSuccess && !s->stream) {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        s->own_stream = true;
    }
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "server stream");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return WAVE2D_OK;
}

int wave2d_server_submit(wave2d_server_t s, const wave2d_request* r) {
    if (!s || !r) return set_error(WAVE2D_ERR_ARG, "null argument");
    if (r->nx < 1 || r->ny < 1 || r->steps < 0 || (r->scheme != 5 && r->scheme != 9 && r->scheme != 13))
        return set_error(WAVE2D_ERR_ARG, "invalid request");
    if ((r->u0 == nullptr) != (r->v0 == nullptr)) return set_error(WAVE2D_ERR_ARG, "u0 and v0 go together");
    if (r->flags & ~(WAVE2D_ALLOW_UNSTABLE | WAVE2D_CONVENTIONAL))
        return set_error(WAVE2D_ERR_ARG, "request flags may hold WAVE2D_ALLOW_UNSTABLE and WAVE2D_CONVENTIONAL only");
    const double lam = r->c * r->tau / r->h;
    if (!(lam > 0) || (lam > wave2d_lambda_max(r->scheme, (r->flags & WAVE2D_CONVENTIONAL) != 0) * (1 + 1e-12) &&
                       !(r->flags & WAVE2D_ALLOW_UNSTABLE)))
        return set_error(WAVE2D_ERR_UNSTABLE, "Courant number outside the stability region");
    if (required_bytes_of(r->nx, r->ny, WAVE2D_F32) > s->budget)
        return set_error(WAVE2D_ERR_OOM, "request larger than the whole device-memory budget");
    Pending p;
    p.r = *r;
    p.t_submit = now_s();
    if (r->u0) {
        const size_t n = (size_t)r->nx * r->ny;
        p.u0.assign(r->u0, r->u0 + n);
        p.v0.assign(r->v0, r->v0 + n);
    }
    p.r.u0 = p.r.v0 = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return set_error(WAVE2D_ERR_STATE, "server is shutting down");
    s->queue.push_back(std::move(p));
    s->submitted += 1;
    s->cv.notify_one();
    return WAVE2D_OK;
}

int wave2d_server_poll(wave2d_server_t s, wave2d_completion* out, int max, int* n_out) {
    if (!s || !n_out || (max > 0 && !out)) return set_error(WAVE2D_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    if (s->fatal) return set_error(s->fatal, "%s", s->fatal_msg.c_str());
    return WAVE2D_OK;
}

int wave2d_server_drain(wave2d_server_t s, double timeout_s) {
    if (!s) return set_error(WAVE2D_ERR_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (s->completed < s->submitted && !s->fatal) {
        if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && s->completed < s->submitted)
            return set_error(WAVE2D_ERR_TIMEOUT, "requests still running after %.1f s", timeout_s);
    }
    if (s->fatal) return set_error(s->fatal, "%s", s->fatal_msg.c_str());
    return WAVE2D_OK;
}

int wave2d_server_stats(wave2d_server_t s, wave2d_server_stats_t* st) {
    if (!s || !st) return set_error(WAVE2D_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->queued = (int64_t)s->queue.size();
    st->node_updates = s->node_updates;
    st->rounds = s->rounds;
    st->used_bytes = s->used;
    st->max_resident_seen = s->max_resident_seen;
    st->gpu_busy_s = s->busy_s;
    return WAVE2D_OK;
}

void wave2d_server_destroy(wave2d_server_t s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
