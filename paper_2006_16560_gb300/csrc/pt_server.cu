// pt_server.cu -- serving loop for long-range kick requests from many
// concurrent simulations (continuous batching).
//
// Each simulation's particle state (positions, velocities, masses, last
// accelerations, potentials and neighbour lists) stays resident in device
// memory between requests.  Several worker threads, each with its own context
// and stream, form batches from the queued requests -- in arrival order, at
// most one request per simulation, skipping simulations that another worker
// has on the GPU (so a simulation's requests run one after the other), within
// a particle cap -- and run each batch as one pass of the pipeline
// (pt_batch_longrange_force over the batch's simulations) between a drift and
// a kick kernel.  Requests that arrive while batches are on the GPU are taken
// by the next worker to become free, and the batches of different workers
// overlap on the device, so a small request does not wait for a large
// simulation's batch to finish.  With two or more workers, half of them
// serve the large simulations on low-priority streams and the others serve
// the rest on high-priority streams: the force kernels run one CTA per group,
// so as the CTAs of a large batch retire the block scheduler starts those of
// the small batches first.  A request's result does not depend on the
// other requests of its batch or on the worker that ran it: every set keeps
// its own tree, lists and summation order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pt.h"

namespace {

constexpr double kWorkspaceBytesPerParticle = 1536.0;   // tree, groups and lists per batch particle
constexpr int kNbPerParticle = 16;                       // neighbour capacity per particle
constexpr int kDefaultWorkers = 4;                       // concurrent batch pipelines
constexpr long long kDefaultLarge = 1ll << 20;           // particles of a "large" simulation
constexpr long long kDefaultBatchCap = 1ll << 22;        // particles per batch (default cap)

struct KickEntry {
    double *pos, *vel;
    const double *acc;
    long long n;
    double dt;
};

// x += v dt (drift) or v += a dt (kick) for every simulation of a batch;
// blockIdx.y selects the simulation.
__global__ void k_drift_kick(const KickEntry *tab, int kick) {
    const KickEntry e = tab[blockIdx.y];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * e.n;
         i += (long long)gridDim.x * blockDim.x) {
        // separately rounded multiply and add (no fused multiply-add), the
        // same arithmetic as a host-side x + v * dt
        if (kick) e.vel[i] = __dadd_rn(e.vel[i], __dmul_rn(e.acc[i], e.dt));
        else e.pos[i] = __dadd_rn(e.pos[i], __dmul_rn(e.vel[i], e.dt));
    }
}

struct Sim {
    bool live = false;
    bool running = false;           // a worker has one of its requests on the GPU
    long long n = 0;
    double r_in = 0, r_out = 0;
    double *pos = nullptr, *vel = nullptr, *mass = nullptr, *acc = nullptr, *pot = nullptr;
    int64_t *nb_off = nullptr;
    int32_t *nb_idx = nullptr;
    long long nb_cap = 0;
    size_t bytes = 0;
    int inflight = 0;               // queued or running requests
};

struct Req {
    int sim;
    double dt_drift, dt_kick;
    double t_submit = 0, t_start = 0, t_done = 0;
    int batch_size = 0;
    long long batch_particles = 0;
    int status = PT_OK;
    bool done = false;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

bool is_dev(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// One batch pipeline: its own context (batch tree, workspace) and stream,
// and the drift / kick tables of its batch (pinned and device copies; drift
// entries first, kick entries after them, uploaded once per batch).
struct Worker {
    int lane = 0;                   // 0: every simulation, 1: large ones, 2: the others
    pt_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    KickEntry *h_tab = nullptr, *d_tab = nullptr;   // 2 x max_sims entries
    std::thread th;
};

struct pt_server {
    std::vector<Worker> workers;
    int device = 0;
    pt_server_config cfg{};
    long long max_batch = 0;
    size_t resident = 0;
    std::vector<Sim> sims;
    std::unordered_map<long long, Req> reqs;
    std::deque<long long> pending;
    long long next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::chrono::steady_clock::time_point t0;
    int tab_cap = 0;
    // totals
    long long batches = 0, served = 0, particles = 0, interactions = 0;
    double busy_s = 0;              // time with at least one batch on the device
    int active = 0;                 // batches on the device
    double busy_since = 0;
    char err[256] = {0};

    long long large = kDefaultLarge;
    bool in_lane(int lane, const Sim &m) const {
        return lane == 0 || (lane == 1) == (m.n >= large);
    }
    bool runnable(int lane) const {   // a queued request of the lane whose simulation is idle (lock held)
        for (long long k : pending) {
            const Sim &m = sims[reqs.at(k).sim];
            if (!m.running && in_lane(lane, m)) return true;
        }
        return false;
    }
    void run(int w);
};

void pt_server::run(int w) {
    cudaSetDevice(device);
    Worker &W = workers[w];
    for (;;) {
        std::vector<long long> batch;
        std::vector<Sim> bs;                      // snapshots: the tables may grow meanwhile
        std::vector<double> dtd, dtk;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return (stop && pending.empty()) || runnable(W.lane); });
            if (stop && pending.empty()) return;
            // continuous batching: arrival order, one request per simulation,
            // simulations on the GPU with another worker skipped (with all of
            // their later requests: each simulation's requests stay in order),
            // and a particle cap; a request that does not fit stays queued for
            // the next batch
            std::vector<char> taken(sims.size(), 0);
            long long np = 0;
            for (auto it = pending.begin(); it != pending.end();) {
                Req &r = reqs[*it];
                Sim &m = sims[r.sim];
                if (taken[r.sim] || m.running || !in_lane(W.lane, m)) { ++it; continue; }
                taken[r.sim] = 1;
                if (!batch.empty() && np + m.n > max_batch) { ++it; continue; }
                np += m.n;
                m.running = true;
                batch.push_back(*it);
                it = pending.erase(it);
            }
            const double t = now_s(t0);
            if (active++ == 0) busy_since = t;
            for (long long k : batch) {
                Req &r = reqs[k];
                r.t_start = t;
                bs.push_back(sims[r.sim]);
                dtd.push_back(r.dt_drift);
                dtk.push_back(r.dt_kick);
            }
        }
        // device work (no lock held: submitters keep queueing meanwhile)
        const int B = (int)batch.size();
        std::vector<pt_cluster_desc> d(B);
        long long np = 0;
        int status = PT_OK;
        for (int k = 0; k < B; k++) {
            const Sim &s = bs[k];
            d[k] = pt_cluster_desc{};
            d[k].n = s.n;
            d[k].pos = s.pos;
            d[k].mass = s.mass;
            d[k].r_in = s.r_in;
            d[k].r_out = s.r_out;
            d[k].acc = s.acc;
            d[k].pot = s.pot;
            d[k].nb_offsets = cfg.neighbours ? s.nb_off : nullptr;
            d[k].nb_idx = cfg.neighbours ? s.nb_idx : nullptr;
            d[k].nb_capacity = cfg.neighbours ? s.nb_cap : 0;
            W.h_tab[k] = KickEntry{s.pos, s.vel, s.acc, s.n, dtd[k]};
            np += s.n;
        }
        // drift entries [0, B), kick entries [B, 2B): one upload; the pinned
        // table is rewritten only after the stream synchronisation below
        for (int k = 0; k < B; k++) {
            W.h_tab[B + k] = W.h_tab[k];
            W.h_tab[B + k].dt = dtk[k];
        }
        cudaMemcpyAsync(W.d_tab, W.h_tab, 2 * B * sizeof(KickEntry), cudaMemcpyHostToDevice, W.stream);
        k_drift_kick<<<dim3(64, B), 256, 0, W.stream>>>(W.d_tab, 0);
        pt_stats st{};
        status = pt_batch_longrange_force(W.ctx, B, d.data(), &cfg.params, 0, &st);
        if (status != PT_OK && status != PT_ERR_CAPACITY) {
            std::lock_guard<std::mutex> lk(mu);
            snprintf(err, sizeof err, "worker %d: %s", w, pt_last_error(W.ctx));
        }
        k_drift_kick<<<dim3(64, B), 256, 0, W.stream>>>(W.d_tab + B, 1);
        if (cudaStreamSynchronize(W.stream) != cudaSuccess) {
            (void)cudaGetLastError();
            status = PT_ERR_CUDA;
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            const double t = now_s(t0);
            if (--active == 0) busy_s += t - busy_since;
            batches++;
            served += B;
            particles += np;
            interactions += st.cell_interactions + st.pp_interactions;
            for (long long k : batch) {
                Req &r = reqs[k];
                r.t_done = t;
                r.batch_size = B;
                r.batch_particles = np;
                r.status = status;
                r.done = true;
                sims[r.sim].inflight--;
                sims[r.sim].running = false;
            }
        }
        cv_done.notify_all();
        cv_work.notify_all();     // the finished simulations' later requests may run now
    }
}

extern "C" {

int pt_server_create(pt_ctx *ctx, const pt_server_config *cfg, pt_server **out) {
    if (!ctx || !cfg || !out) return PT_ERR_ARG;
    *out = nullptr;
    if (cfg->hbm_budget_bytes == 0 || cfg->max_sims < 1 || cfg->workers < 0 || cfg->workers > 16) return PT_ERR_ARG;
    pt_server *s = new (std::nothrow) pt_server;
    if (!s) return PT_ERR_OOM;
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return PT_ERR_CUDA;
    }
    const int nw = cfg->workers > 0 ? cfg->workers : kDefaultWorkers;
    // every worker keeps a batch workspace: half the budget is theirs
    const double room = (double)cfg->hbm_budget_bytes / 2.0 / nw / kWorkspaceBytesPerParticle;
    s->max_batch = cfg->max_batch_particles > 0 ? cfg->max_batch_particles
                                                : (long long)std::min(room, (double)kDefaultBatchCap);
    s->tab_cap = cfg->max_sims;
    s->large = cfg->large_sim_particles > 0 ? cfg->large_sim_particles : kDefaultLarge;
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        (void)cudaGetLastError();
        prio_low = prio_high = 0;
    }
    s->workers.resize(nw);
    for (int w = 0; w < nw; w++) {
        Worker &W = s->workers[w];
        W.lane = nw == 1 ? 0 : (w < nw / 2 ? 1 : 2);
        if (cudaStreamCreateWithPriority(&W.stream, cudaStreamNonBlocking, W.lane == 1 ? prio_low : prio_high) !=
                cudaSuccess ||
            cudaMallocHost((void **)&W.h_tab, 2 * s->tab_cap * sizeof(KickEntry)) != cudaSuccess ||
            cudaMalloc((void **)&W.d_tab, 2 * s->tab_cap * sizeof(KickEntry)) != cudaSuccess) {
            (void)cudaGetLastError();
            pt_server_destroy(s);
            return PT_ERR_OOM;
        }
        const int rc = pt_ctx_create(&W.ctx, s->device, W.stream);
        if (rc != PT_OK) {
            pt_server_destroy(s);
            return rc;
        }
    }
    s->t0 = std::chrono::steady_clock::now();
    for (int w = 0; w < nw; w++) s->workers[w].th = std::thread([s, w] { s->run(w); });
    *out = s;
    return PT_OK;
}

int pt_server_destroy(pt_server *s) {
    if (!s) return PT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (Worker &W : s->workers)
        if (W.th.joinable()) W.th.join();
    cudaSetDevice(s->device);
    for (Sim &m : s->sims)
        if (m.live) {
            cudaFree(m.pos); cudaFree(m.vel); cudaFree(m.mass); cudaFree(m.acc); cudaFree(m.pot);
            cudaFree(m.nb_off); cudaFree(m.nb_idx);
        }
    for (Worker &W : s->workers) {
        if (W.h_tab) cudaFreeHost(W.h_tab);
        if (W.d_tab) cudaFree(W.d_tab);
        if (W.ctx) pt_ctx_destroy(W.ctx);
        if (W.stream) cudaStreamDestroy(W.stream);
    }
    delete s;
    return PT_OK;
}

int pt_server_add_sim(pt_server *s, int64_t n, const double *pos, const double *vel,
                      const double *mass, double r_in, double r_out, int *sim_id) {
    if (!s || !sim_id || n < 1 || !pos || !vel || !mass) return PT_ERR_ARG;
    if (!(r_in >= 0.0) || !(r_out > r_in)) return PT_ERR_ARG;
    if (n > s->max_batch) return PT_ERR_CAPACITY;
    const long long nbc = kNbPerParticle * n + 64;
    const size_t bytes = (size_t)n * (24 + 24 + 8 + 24 + 8 + 8) + 8 + (size_t)nbc * 4;
    std::lock_guard<std::mutex> lk(s->mu);
    const double reserve = kWorkspaceBytesPerParticle * (double)s->max_batch * (double)s->workers.size();
    if ((double)(s->resident + bytes) + reserve > (double)s->cfg.hbm_budget_bytes) return PT_ERR_CAPACITY;
    int id = -1;
    for (size_t k = 0; k < s->sims.size(); k++)
        if (!s->sims[k].live && s->sims[k].inflight == 0) { id = (int)k; break; }
    if (id < 0) {
        if ((int)s->sims.size() >= s->cfg.max_sims) return PT_ERR_CAPACITY;
        s->sims.emplace_back();
        id = (int)s->sims.size() - 1;
    }
    Sim m;
    m.n = n;
    m.r_in = r_in;
    m.r_out = r_out;
    m.nb_cap = nbc;
    m.bytes = bytes;
    cudaSetDevice(s->device);
    if (cudaMalloc((void **)&m.pos, n * 24) != cudaSuccess || cudaMalloc((void **)&m.vel, n * 24) != cudaSuccess ||
        cudaMalloc((void **)&m.mass, n * 8) != cudaSuccess || cudaMalloc((void **)&m.acc, n * 24) != cudaSuccess ||
        cudaMalloc((void **)&m.pot, n * 8) != cudaSuccess ||
        cudaMalloc((void **)&m.nb_off, (n + 1) * 8) != cudaSuccess ||
        cudaMalloc((void **)&m.nb_idx, nbc * 4) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(m.pos); cudaFree(m.vel); cudaFree(m.mass); cudaFree(m.acc); cudaFree(m.pot);
        cudaFree(m.nb_off); cudaFree(m.nb_idx);
        return PT_ERR_OOM;
    }
    const cudaMemcpyKind k1 = is_dev(pos) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind k2 = is_dev(vel) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind k3 = is_dev(mass) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpy(m.pos, pos, n * 24, k1) != cudaSuccess || cudaMemcpy(m.vel, vel, n * 24, k2) != cudaSuccess ||
        cudaMemcpy(m.mass, mass, n * 8, k3) != cudaSuccess) {
        (void)cudaGetLastError();
        return PT_ERR_CUDA;
    }
    m.live = true;
    s->sims[id] = m;
    s->resident += bytes;
    *sim_id = id;
    return PT_OK;
}

int pt_server_remove_sim(pt_server *s, int sim_id) {
    if (!s) return PT_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (sim_id < 0 || sim_id >= (int)s->sims.size() || !s->sims[sim_id].live) return PT_ERR_ARG;
    s->cv_done.wait(lk, [&] { return s->sims[sim_id].inflight == 0; });
    Sim &m = s->sims[sim_id];
    cudaSetDevice(s->device);
    cudaFree(m.pos); cudaFree(m.vel); cudaFree(m.mass); cudaFree(m.acc); cudaFree(m.pot);
    cudaFree(m.nb_off); cudaFree(m.nb_idx);
    s->resident -= m.bytes;
    m = Sim{};
    return PT_OK;
}

int pt_server_submit(pt_server *s, int sim_id, double dt_drift, double dt_kick, int64_t *ticket) {
    if (!s || !ticket) return PT_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (sim_id < 0 || sim_id >= (int)s->sims.size() || !s->sims[sim_id].live) return PT_ERR_ARG;
        const long long t = s->next_ticket++;
        Req r;
        r.sim = sim_id;
        r.dt_drift = dt_drift;
        r.dt_kick = dt_kick;
        r.t_submit = now_s(s->t0);
        s->reqs.emplace(t, r);
        s->pending.push_back(t);
        s->sims[sim_id].inflight++;
        *ticket = t;
    }
    s->cv_work.notify_all();      // workers of different lanes wait on this variable
    return PT_OK;
}

int pt_server_wait(pt_server *s, int64_t ticket, double timeout_s, pt_request_info *info) {
    if (!s) return PT_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return PT_ERR_ARG;
    const auto pred = [&] { return s->reqs[ticket].done; };
    if (timeout_s < 0) s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return PT_ERR_TIMEOUT;
    const Req &r = s->reqs[ticket];
    if (info) {
        info->ticket = ticket;
        info->sim = r.sim;
        info->t_submit = r.t_submit;
        info->t_start = r.t_start;
        info->t_done = r.t_done;
        info->batch_size = r.batch_size;
        info->batch_particles = r.batch_particles;
        info->status = r.status;
    }
    const int st = r.status;
    s->reqs.erase(ticket);
    return st == PT_ERR_CAPACITY ? PT_OK : st;     // neighbour overflow keeps acc / pot valid
}

int pt_server_read_sim(pt_server *s, int sim_id, double *pos, double *vel, double *acc, double *pot) {
    if (!s) return PT_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (sim_id < 0 || sim_id >= (int)s->sims.size() || !s->sims[sim_id].live) return PT_ERR_ARG;
    s->cv_done.wait(lk, [&] { return s->sims[sim_id].inflight == 0; });
    const Sim &m = s->sims[sim_id];
    cudaSetDevice(s->device);
    struct { void *dst; const void *src; size_t b; } cp[4] = {
        {pos, m.pos, (size_t)m.n * 24}, {vel, m.vel, (size_t)m.n * 24},
        {acc, m.acc, (size_t)m.n * 24}, {pot, m.pot, (size_t)m.n * 8}};
    for (auto &c : cp)
        if (c.dst && cudaMemcpy(c.dst, c.src, c.b, cudaMemcpyDefault) != cudaSuccess) {
            (void)cudaGetLastError();
            return PT_ERR_CUDA;
        }
    return PT_OK;
}

const char *pt_server_last_error(pt_server *s) { return s ? s->err : "no server"; }

int pt_server_stats(pt_server *s, pt_server_stats_t *out) {
    if (!s || !out) return PT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->batches = s->batches;
    out->requests = s->served;
    out->particles = s->particles;
    out->interactions = s->interactions;
    out->busy_s = s->busy_s;
    out->uptime_s = now_s(s->t0);
    out->resident_bytes = (int64_t)s->resident;
    out->max_batch_particles = s->max_batch;
    out->queued = (int64_t)s->pending.size();
    return PT_OK;
}

}  // extern "C"
