// Continuous-batching run server.
//
// Requests are complete runs (model, lattice, tau, steps, initial state).
// Runs go to one of two lanes by their estimated step cost: small runs and
// large runs (a step of a 2048^2 16-velocity FD lattice or more). Each lane
// is a worker thread owning a dynamic Engine on its own CUDA stream, the
// small-run lane's at the device's highest stream priority and the large-run
// lane's at the lowest: both lanes' kernels run on the GPU at the same time,
// the small runs' blocks are dispatched first as SMs free up (the large
// lane launches many short blocks, so SMs free up every few tens of
// microseconds), and the large runs use the rest, so a large run is not held
// back by the rounds of the
// small ones (nor they by its long steps). A lane admits queued requests of
// its class as slots and device memory (an HBM budget on the summed lattice
// footprints of both lanes) free up, advances its resident runs together in
// rounds that give each run about the same device time (the cheapest run
// advances its lane's chunk of steps, costlier ones proportionally fewer; one
// captured CUDA-graph replay per 32 steps, runs that have spent their
// allotment are skipped by the kernels), and retires finished runs at the end
// of a round: final observables, recorded series, fitted apparent viscosity,
// then the lattice's memory is released and waiting requests are admitted.
// Requests that arrive while others are on the GPU join at their lane's next
// round. With a caller's stream the server runs one lane on it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Req {
    lbm_request r{};
    double t_submit = 0, t_admit = -1, t_done = -1;
    int state = 0;  // 0 queued, 1 running, 2 done
    int lat = -1;
    long long left = 0;  // steps still to run (worker thread only)
    size_t bytes = 0;
    bool cancel = false;
    int lane = 0;        // 0 small runs, 1 large runs
    lbm_result res{};
    std::vector<lbm_obs> series;
    std::vector<double> rho, ux, uy;   // final fields (keep_moments)
};

// Initial fields of a request (Sec. 4.1-4.3 set-ups), node coordinates
// x_i = i, one wavelength across the lattice.
void initial_fields(const lbm_request& q, std::vector<double>& rho, std::vector<double>& ux, std::vector<double>& uy) {
    const int nx = q.spec.nx, ny = q.spec.ny;
    const size_t n = (size_t)nx * ny;
    rho.assign(n, 1.0);
    ux.assign(n, 0.0);
    uy.assign(n, 0.0);
    const double rho0 = q.spec.rho0 > 0 ? q.spec.rho0 : 1.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t c = (size_t)y * nx + x;
            const double kx = 2 * kPi * x / nx, ky = 2 * kPi * y / ny;
            if (q.init == 0) {  // Taylor-Green, pressure-balanced density (cs = 1)
                ux[c] = q.U * std::sin(kx) * std::cos(ky);
                uy[c] = -q.U * std::cos(kx) * std::sin(ky);
                rho[c] = rho0 * (1.0 + q.U * q.U / 4.0 * (std::cos(2 * kx) + std::cos(2 * ky)));
            } else if (q.init == 1) {  // shear wave
                rho[c] = rho0;
                uy[c] = q.U * std::sin(kx);
            } else {  // shock tube
                rho[c] = x <= nx / 2 ? q.rho_l : q.rho_r;
            }
        }
}

// Estimated device time of one step of a run alone, for sharing the device
// between runs: about 20 us of fixed cost per step (launch and tile latency
// of a small lattice) plus a cost per node, from single-lattice rates on
// GB300 (FP32: CS D2Q9 in place 74 GLUPS, FD 16-velocity 4.4 GLUPS, the FD
// cost scaled by the number of velocities; FP64 on the narrow FP64 pipe; an
// FD step with the IMEX scheme 1.1x, temporally blocked 3.0x the RK3 step,
// as measured for FD 16-velocity 4096^2). Only the ratios between runs matter.
double step_cost(const lbm_spec& s) {
    const double nodes = (double)s.nx * s.ny;
    const double k = (double)s.q_per_axis * s.q_per_axis;
    const double scheme = s.model == LBM_CS ? 1.0
                          : (s.scheme == LBM_TS_IMEX ? 1.1 : (s.scheme == LBM_TS_RK3_FUSED ? 3.0 : 1.0));
    const double per_node = s.model == LBM_CS ? (s.precision == LBM_FP64 ? 0.125e-9 : 0.0135e-9)
                                              : (s.precision == LBM_FP64 ? 6e-9 : 0.227e-9) * k / 16.0 * scheme;
    return 20e-6 + nodes * per_node;
}

// Steps of one scheduling round (see lbm_server_create): the run with the
// cheapest step advances `chunk` steps, a run whose step costs m times as
// much chunk / m (at least one), none more than it has left.
void plan_round(const double* cost, const long long* left, size_t n, int chunk, long long* steps) {
    double cmin = 1e300;
    for (size_t i = 0; i < n; ++i) cmin = std::min(cmin, cost[i]);
    for (size_t i = 0; i < n; ++i) {
        const long long share = std::max(1LL, std::llround(chunk * cmin / cost[i]));
        steps[i] = std::min(std::min<long long>(chunk, share), left[i]);
    }
}

// Runs whose estimated step (step_cost) takes this long or longer go to the
// large-run lane: FD 16-velocity FP32 from 2048^2 (~1 ms), CS FP32 from
// about 6000^2.
constexpr double kLargeStepCost = 0.5e-3;

// A lane: a worker thread with its engine, its stream and its runs.
struct Lane {
    lbm::Engine e;
    std::thread worker;
    std::deque<uint64_t> queue;     // guarded by the server's mutex
    std::vector<uint64_t> running;  // worker thread only
    int inject_applied = 0;         // worker thread only
    int chunk = 1;
    cudaStream_t stream = nullptr;  // created by the server (null: the caller's stream)
};

}  // namespace

struct lbm_server {
    Lane lanes[2];
    int n_lanes = 2;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    size_t budget = 0, resident = 0;
    int resident_runs = 0;          // admitted and not finished, both lanes (guarded by mu)
    int max_slots = 1, chunk = 256;
    uint64_t next_ticket = 1;
    std::map<uint64_t, Req> reqs;
    int64_t n_done = 0;
    std::atomic<int> inject_req{0};  // wait-timeout injection requested (microseconds, 0 = off)
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }

    void finish(Req& q, int status) {  // caller holds mu
        if (q.state == 1) --resident_runs;
        q.state = 2;
        q.t_done = now();
        q.res.status = status;
        q.res.user_tag = q.r.user_tag;
        q.res.t_submit = q.t_submit;
        q.res.t_admit = q.t_admit;
        q.res.t_done = q.t_done;
        q.res.n_series = (int64_t)q.series.size();
        ++n_done;
        cv_done.notify_all();
        cv_work.notify_all();   // slots or memory may have freed up for the other lane
    }

    // Set-up of an admitted request on its lane's worker thread (no lock held).
    int start(lbm::Engine& e, Req& q) {
        int idx = -1;
        int rc = e.add_lattice(&q.r.spec, &idx);
        if (rc) return rc;
        q.lat = idx;
        std::vector<double> rho, ux, uy;
        initial_fields(q.r, rho, ux, uy);
        rc = e.init(idx, rho.data(), ux.data(), uy.data());
        if (rc) return rc;
        const int nx = q.r.spec.nx, ny = q.r.spec.ny;
        if (q.r.init == 0 || q.r.init == 1) {
            std::vector<double> px(nx), py(ny);
            for (int x = 0; x < nx; ++x) px[x] = std::sin(2 * kPi * x / nx);
            for (int y = 0; y < ny; ++y) py[y] = q.r.init == 0 ? std::cos(2 * kPi * y / ny) : 1.0;
            rc = e.set_probe(idx, q.r.init == 0 ? 0 : 1, px.data(), py.data(),
                             (q.r.init == 0 ? 4.0 : 2.0) / ((double)nx * ny));
            if (rc) return rc;
        }
        rc = e.observables(idx, &q.res.first);
        if (rc) return rc;
        if (q.r.obs_every > 0) {
            rc = e.record(idx, q.r.obs_every, q.r.steps / q.r.obs_every + 1);
            if (rc) return rc;
        }
        rc = e.release_io(idx);  // only the state stays resident (the budget counts it)
        if (rc) return rc;
        q.left = q.r.steps;
        return e.set_budget(idx, 0);  // steps are allotted round by round
    }

    // Results of a run whose budget is exhausted (worker thread, no lock).
    int collect(lbm::Engine& e, Req& q) {
        int rc = e.observables(q.lat, &q.res.last);
        if (rc) return rc;
        if (q.r.keep_moments) {
            const size_t n = (size_t)q.r.spec.nx * q.r.spec.ny;
            q.rho.resize(n);
            q.ux.resize(n);
            q.uy.resize(n);
            rc = e.moments(q.lat, q.rho.data(), q.ux.data(), q.uy.data());
            if (rc) return rc;
        }
        q.res.steps = e.L(q.lat).step0;
        if (q.r.obs_every > 0) {
            long long n = 0;
            rc = e.series(q.lat, nullptr, 0, &n);
            if (rc) return rc;
            q.series.resize((size_t)n);
            if (n) rc = e.series(q.lat, q.series.data(), n, &n);
            if (rc) return rc;
        }
        q.res.nu_fit = 0;
        if ((q.r.init == 0 || q.r.init == 1) && q.series.size() >= 4) {
            // decay of the projected amplitude, Eq. (shear_sol) / Eq. (taylor):
            // A ~ exp(-m k^2 nu t), m = 1 (shear) or 2 (Taylor-Green)
            std::vector<double> t, a;
            for (const auto& o : q.series) {
                t.push_back(o.time);
                a.push_back(o.amp);
            }
            double gamma = 0, a0 = 0;
            const double skip = 0.1 * t.back();
            if (lbm_fit_decay(t.data(), a.data(), (int64_t)t.size(), skip, &gamma, &a0) == LBM_OK) {
                const double L = q.r.spec.nx * e.L(q.lat).spec.dx;
                const double k = 2 * kPi / L;
                q.res.nu_fit = gamma / ((q.r.init == 0 ? 2.0 : 1.0) * k * k);
            }
        }
        return q.res.last.nonfinite ? LBM_ENONFINITE : LBM_OK;
    }

    void loop(int li) {
        Lane& ln = lanes[li];
        lbm::Engine& e = ln.e;
        std::vector<uint64_t>& running = ln.running;
        for (;;) {
            std::vector<uint64_t> admit;
            {
                std::unique_lock<std::mutex> lk(mu);
                for (;;) {
                    // admission: oldest first, skipping requests that do not
                    // fit yet (first fit over the lane's queue); slots and
                    // memory are shared by the lanes
                    for (auto it = ln.queue.begin(); it != ln.queue.end();) {
                        Req& q = reqs[*it];
                        if (resident_runs >= max_slots) break;
                        if (resident + q.bytes <= budget) {
                            resident += q.bytes;
                            ++resident_runs;
                            q.state = 1;
                            q.t_admit = now();
                            admit.push_back(*it);
                            it = ln.queue.erase(it);
                        } else {
                            ++it;
                        }
                    }
                    if (!admit.empty() || !running.empty() || stop) break;
                    cv_work.wait(lk);
                }
                if (stop && admit.empty() && running.empty()) return;
            }
            for (uint64_t t : admit) {
                Req* q;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    q = &reqs[t];
                }
                const int rc = start(e, *q);
                std::lock_guard<std::mutex> lk(mu);
                if (rc) {
                    if (q->lat >= 0) e.remove_lattice(q->lat);
                    resident -= q->bytes;
                    finish(*q, rc);
                } else {
                    running.push_back(t);
                }
            }
            if (running.empty()) continue;
            int rc = LBM_OK;
            const int want = inject_req.load();
            if (want != ln.inject_applied) {
                rc = e.inject_wait_timeout(want);
                ln.inject_applied = want;
            }
            // One round: every resident run gets about the same device time.
            // The cheapest run (by step_cost) advances `chunk` steps, a run
            // whose step costs m times as much advances chunk / m steps (at
            // least one), none more than it has left. Runs that finish their
            // allotment early sit out the rest of the round.
            std::vector<Req*> rq;
            {
                std::lock_guard<std::mutex> lk(mu);
                for (uint64_t t : running) rq.push_back(&reqs[t]);
            }
            std::vector<long long> steps(rq.size(), 0);
            long long round_steps = 0;
            if (rc == LBM_OK) {
                std::vector<double> cost(rq.size());
                std::vector<long long> left(rq.size());
                for (size_t i = 0; i < rq.size(); ++i) {
                    cost[i] = step_cost(rq[i]->r.spec);
                    left[i] = rq[i]->left;
                }
                plan_round(cost.data(), left.data(), rq.size(), ln.chunk, steps.data());
                std::vector<std::pair<int, long long>> budgets;
                for (size_t i = 0; i < rq.size(); ++i) {
                    round_steps = std::max(round_steps, steps[i]);
                    budgets.emplace_back(rq[i]->lat, steps[i]);
                }
                rc = e.set_budgets(budgets);
            }
            if (rc == LBM_OK) rc = e.step(round_steps);
            if (rc == LBM_OK) rc = e.sync();
            std::vector<uint64_t> still;
            for (size_t i = 0; i < rq.size(); ++i) {
                const uint64_t t = running[i];
                Req* q = rq[i];
                bool cancel;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    cancel = q->cancel || stop;
                }
                if (rc == LBM_OK) q->left -= steps[i];
                if (rc == LBM_OK && !cancel && q->left > 0) {
                    still.push_back(t);
                    continue;
                }
                int st = rc;
                if (st == LBM_OK && !cancel) st = collect(e, *q);
                else if (st == LBM_OK) st = LBM_ECANCELLED;
                e.remove_lattice(q->lat);
                std::lock_guard<std::mutex> lk(mu);
                resident -= q->bytes;
                finish(*q, st);
            }
            running.swap(still);
        }
    }
};

extern "C" {

int lbm_server_create(lbm_server** out, size_t hbm_budget_bytes, int max_slots, int chunk_steps, void* stream) {
    try {
        if (!out || hbm_budget_bytes == 0 || max_slots < 1 || chunk_steps < 1) {
            lbm::set_error("server needs a budget, at least one slot and a positive chunk");
            return LBM_EINVAL;
        }
        *out = nullptr;
        lbm_server* s = new lbm_server;
        s->budget = hbm_budget_bytes;
        s->max_slots = max_slots;
        s->chunk = chunk_steps;
        s->n_lanes = stream ? 1 : 2;
        int lo = 0, hi = 0;   // stream priorities: numerically lower is higher
        cudaError_t e_streams = cudaSuccess;
        if (!stream) {
            cudaError_t& e = e_streams;
            e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->lanes[0].stream, cudaStreamNonBlocking, hi);
            if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->lanes[1].stream, cudaStreamNonBlocking, lo);
        }
        // on failure: the engines go first (they finish their streams), then the streams
        auto fail = [s](int rc) {
            cudaStream_t st[2] = {s->lanes[0].stream, s->lanes[1].stream};
            delete s;
            for (cudaStream_t x : st)
                if (x) cudaStreamDestroy(x);
            return rc;
        };
        if (e_streams != cudaSuccess) return fail(lbm::cuda_fail(e_streams, "server streams"));
        for (int li = 0; li < s->n_lanes; ++li) {
            Lane& ln = s->lanes[li];
            ln.e.dynamic_ = true;
            ln.chunk = li == 0 ? chunk_steps : std::max(1, chunk_steps / 8);
            // Blocks of a running kernel are not preempted: stream priority
            // only decides which stream's blocks fill SMs as they free up. A
            // large lane of one block set per SM holds every SM for a whole
            // launch (an FD 4096^2 stage: 1.1 ms) and the small lane waits
            // that long for each of its steps; with 16 block sets, each
            // block covers a few tiles (about 70 us of that stage).
            if (li == 1) ln.e.grid_mult_ = 16;
            const int rc = ln.e.open(stream ? stream : ln.stream);
            if (rc) return fail(rc);
        }
        for (int li = 0; li < s->n_lanes; ++li) s->lanes[li].worker = std::thread([s, li] { s->loop(li); });
        *out = s;
        return LBM_OK;
    } catch (...) {
        lbm::set_error("server creation failed");
        return LBM_ENOMEM;
    }
}

int lbm_submit(lbm_server* s, const lbm_request* req, uint64_t* ticket) {
    try {
        if (!s || !req || !ticket) return LBM_EINVAL;
        lbm_spec spec;
        int rc = lbm::Engine::validate(&req->spec, &spec);
        if (rc) return rc;
        if (req->steps < 0 || req->init < 0 || req->init > 2 || req->obs_every < 0 || !std::isfinite(req->U) ||
            (req->init == 2 && !(req->rho_l > 0 && req->rho_r > 0))) {
            lbm::set_error("bad request (steps, init, obs_every, U or shock densities)");
            return LBM_EINVAL;
        }
        const size_t bytes = lbm::Engine::footprint(spec);
        std::lock_guard<std::mutex> lk(s->mu);
        if (bytes > s->budget) {
            lbm::set_error("request can never fit the server's memory budget");
            return LBM_ENOMEM;
        }
        const uint64_t t = s->next_ticket++;
        Req& q = s->reqs[t];
        q.r = *req;
        q.r.spec = spec;
        q.bytes = bytes;
        q.t_submit = s->now();
        q.lane = (s->n_lanes > 1 && step_cost(spec) >= kLargeStepCost) ? 1 : 0;
        s->lanes[q.lane].queue.push_back(t);
        *ticket = t;
        s->cv_work.notify_all();
        return LBM_OK;
    } catch (...) {
        lbm::set_error("submit failed");
        return LBM_ENOMEM;
    }
}

int lbm_poll(lbm_server* s, uint64_t ticket, lbm_result* out) {
    if (!s || !out) return LBM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LBM_ENOTFOUND;
    if (it->second.state != 2) return LBM_ENOTREADY;
    *out = it->second.res;
    return LBM_OK;
}

int lbm_result_series(lbm_server* s, uint64_t ticket, lbm_obs* out, int64_t cap, int64_t* count) {
    if (!s || cap < 0 || (cap > 0 && !out)) return LBM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LBM_ENOTFOUND;
    if (it->second.state != 2) return LBM_ENOTREADY;
    const auto& v = it->second.series;
    if (count) *count = (int64_t)v.size();
    for (int64_t i = 0; i < cap && i < (int64_t)v.size(); ++i) out[i] = v[i];
    return LBM_OK;
}

int lbm_result_moments(lbm_server* s, uint64_t ticket, double* rho, double* ux, double* uy) {
    if (!s || !rho || !ux || !uy) return LBM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LBM_ENOTFOUND;
    const Req& q = it->second;
    if (q.state != 2) return LBM_ENOTREADY;
    const size_t n = (size_t)q.r.spec.nx * q.r.spec.ny;
    if (q.rho.size() != n) {
        lbm::set_error("no kept fields for this ticket (request without keep_moments, or the run failed)");
        return LBM_ENOTFOUND;
    }
    std::copy(q.rho.begin(), q.rho.end(), rho);
    std::copy(q.ux.begin(), q.ux.end(), ux);
    std::copy(q.uy.begin(), q.uy.end(), uy);
    return LBM_OK;
}

int lbm_release(lbm_server* s, uint64_t ticket) {
    if (!s) return LBM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LBM_ENOTFOUND;
    if (it->second.state != 2) return LBM_ENOTREADY;
    s->reqs.erase(it);
    --s->n_done;   // finished results still held
    return LBM_OK;
}

int lbm_cancel(lbm_server* s, uint64_t ticket) {
    if (!s) return LBM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return LBM_ENOTFOUND;
    Req& q = it->second;
    if (q.state == 0) {
        auto& queue = s->lanes[q.lane].queue;
        for (auto qi = queue.begin(); qi != queue.end(); ++qi)
            if (*qi == ticket) {
                queue.erase(qi);
                break;
            }
        s->finish(q, LBM_ECANCELLED);
    } else if (q.state == 1) {
        q.cancel = true;
    }
    return LBM_OK;
}

int lbm_server_plan_round(const lbm_spec* specs, const int64_t* left, int n, int chunk_steps, int64_t* steps) {
    if (n < 0 || chunk_steps < 1 || (n > 0 && (!specs || !left || !steps))) {
        lbm::set_error("plan_round needs n >= 0, chunk_steps >= 1 and the arrays");
        return LBM_EINVAL;
    }
    try {
        std::vector<double> cost((size_t)n);
        std::vector<long long> l((size_t)n), out((size_t)n);
        for (int i = 0; i < n; ++i) {
            lbm_spec norm;
            const int rc = lbm::Engine::validate(&specs[i], &norm);
            if (rc) return rc;
            if (left[i] < 0) {
                lbm::set_error("negative steps left");
                return LBM_EINVAL;
            }
            cost[(size_t)i] = step_cost(norm);
            l[(size_t)i] = left[i];
        }
        plan_round(cost.data(), l.data(), (size_t)n, chunk_steps, out.data());
        for (int i = 0; i < n; ++i) steps[i] = out[(size_t)i];
        return LBM_OK;
    } catch (...) {
        lbm::set_error("plan_round failed");
        return LBM_ENOMEM;
    }
}

int lbm_footprint(const lbm_spec* spec, size_t* bytes) {
    if (!spec || !bytes) {
        lbm::set_error("lbm_footprint needs a spec and an output");
        return LBM_EINVAL;
    }
    lbm_spec norm;
    const int rc = lbm::Engine::validate(spec, &norm);
    if (rc) return rc;
    *bytes = lbm::Engine::footprint(norm);
    return LBM_OK;
}

int lbm_server_inject_wait_timeout(lbm_server* s, int microseconds) {
    if (!s || microseconds < 0 || microseconds > 1000000) {
        lbm::set_error("wait-timeout injection takes 0 (off) to 1e6 microseconds");
        return LBM_EINVAL;
    }
    s->inject_req.store(microseconds);
    return LBM_OK;
}

int lbm_server_drain(lbm_server* s, double timeout_s) {
    if (!s) return LBM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (s->n_done < (int64_t)s->reqs.size()) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->n_done < (int64_t)s->reqs.size()) {
            lbm::set_error("drain timed out");
            return LBM_ETIMEOUT;
        }
    }
    return LBM_OK;
}

int lbm_server_stats(lbm_server* s, int64_t* queued, int64_t* running, int64_t* finished, size_t* resident_bytes) {
    if (!s) return LBM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t nq = (int64_t)(s->lanes[0].queue.size() + s->lanes[1].queue.size());
    if (queued) *queued = nq;
    if (running) *running = (int64_t)s->reqs.size() - nq - s->n_done;
    if (finished) *finished = s->n_done;
    if (resident_bytes) *resident_bytes = s->resident;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& ln : s->lanes) {
            for (uint64_t t : ln.queue) s->finish(s->reqs[t], LBM_ECANCELLED);
            ln.queue.clear();
        }
        s->cv_work.notify_all();
    }
    for (auto& ln : s->lanes)
        if (ln.worker.joinable()) ln.worker.join();
    cudaStream_t streams[2] = {s->lanes[0].stream, s->lanes[1].stream};
    delete s;   // the engines finish and release their work first
    for (cudaStream_t st : streams)
        if (st) cudaStreamDestroy(st);
}

}  // extern "C"
