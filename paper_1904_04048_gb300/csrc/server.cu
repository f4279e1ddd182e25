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
};

}  // namespace
}  // namespace w2d

using namespace w2d;

struct wave2d_server {
    int64_t budget = 0;
    int max_resident = 0;
    int quantum = 64;
    int Tq = 4, OH = 32;
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

// One scheduling round; returns false when there is nothing to do.
bool round_once(wave2d_server* s) {
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
            s->used += need;
            admitted.push_back(std::move(a));
            s->queue.pop_front();
        }
    }
    if (admitted.empty() && s->resident.empty()) return false;

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
            if (rc != WAVE2D_OK) fail_round(s, rc);
        }
        if (!hs_pulse.empty()) {
            size_t total = 0;
            for (Active* a : pulses) total += 2 * (size_t)a->p.r.nx * a->p.r.ny;
            Allocator al = current_allocator();
            double* stage = (double*)dev_alloc(al, total * sizeof(double), s->stream);
            if (!stage) {
                fail_round(s, set_error(WAVE2D_ERR_OOM, "initial-data staging allocation failed"));
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
                dev_free(al, stage, total * sizeof(double), s->stream);
                if (rc != WAVE2D_OK) fail_round(s, rc);
            }
        }
        int64_t first_nodes = 0;
        for (Active& a : admitted) {
            first_nodes += (int64_t)a.p.r.nx * a.p.r.ny;
            s->resident.push_back(std::move(a));
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->node_updates += first_nodes;  // the first level of each request
        s->max_resident_seen = std::max<int>(s->max_resident_seen, (int)s->resident.size());
    }
    if (s->resident.empty()) return true;

    // 3. advance every resident simulation by up to one quantum
    std::vector<wave2d_t> hs;
    std::vector<int64_t> steps;
    for (Active& a : s->resident) {
        hs.push_back(a.h);
        steps.push_back(std::min<int64_t>(a.remaining, s->quantum));
    }
    int64_t nodes = 0;
    for (size_t i = 0; i < hs.size(); ++i) nodes += (int64_t)s->resident[i].p.r.nx * s->resident[i].p.r.ny * steps[i];
    {
        wave2d_tune opt{};
        opt.use_graph = 0;
        opt.temporal_t = s->Tq;
        opt.tile_h = s->OH;
        wave2d_batch_t b = nullptr;
        int rc = wave2d_batch_create(hs.data(), (int)hs.size(), &opt, &b);
        if (rc == WAVE2D_OK) rc = wave2d_batch_run(b, steps.data());
        wave2d_batch_destroy(b);  // synchronises the stream
        if (rc != WAVE2D_OK) fail_round(s, rc);
    }

    // 4. retire finished simulations
    std::vector<Active> still;
    for (size_t i = 0; i < s->resident.size(); ++i) {
        Active& a = s->resident[i];
        a.remaining -= steps[i];
        if (a.remaining > 0) {
            still.push_back(std::move(a));
            continue;
        }
        double l2 = NAN, linf = NAN;
        int rc = wave2d_error_vs_exact(a.h, nullptr, &l2, &linf, nullptr);
        if (a.p.r.out_field && (rc == WAVE2D_OK || rc == WAVE2D_ERR_NONFINITE))
            wave2d_get_state(a.h, nullptr, a.p.r.out_field, nullptr);
        int64_t k = 0;
        wave2d_info_t info;
        if (wave2d_get_info(a.h, &info) == WAVE2D_OK) k = info.k;
        wave2d_destroy(a.h);
        a.h = nullptr;
        complete(s, a, rc, l2, linf, k);
    }
    s->resident.swap(still);
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
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->queue.empty() && s->resident.empty()) break;
            if (s->queue.empty() && s->resident.empty()) {
                s->cv.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        round_once(s);
    }
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
    if (opt && opt->temporal_t >= 1 && opt->temporal_t <= 4) s->Tq = opt->temporal_t;
    if (opt && (opt->tile_h == 32 || opt->tile_h == 64)) s->OH = opt->tile_h;
    cudaError_t e = cudaGetDevice(&s->device);
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
