// Serving loop: continuous batching of independent solves (include/acs.h).
//
// One worker thread per server owns the device side.  Requests are prepared
// on the submitting thread (validation, relabelled rows, sliced-ELLPACK
// images -- the same preparation as a single problem), queued, and admitted
// by the worker when a slot and a block of the device pool are free (first
// fit over one allocation of the budget).  Each round is one cooperative
// launch of the team kernel over every admitted request with a device-side
// deadline: a team that takes a request runs Algorithm 2 on it until it
// converges, reaches its iteration limit, or the deadline passes (checked at
// the end of each iteration, reduced over the team so that its CTAs agree),
// and then takes the next request until the deadline.  Everything a paused
// request needs lives in its pool block (iterates, solver vectors, control
// block, and the cached dense factor when it uses one), so the next round
// resumes it exactly.  Finished requests are copied out and freed between
// rounds.  Requests with more than large_nnz nonzeros run alone on the whole
// GPU through the single-problem launch, between rounds.

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "acs_team.cuh"

namespace acs {
namespace {

using Clock = std::chrono::steady_clock;

// First fit over [0, cap) in 256-byte granules, with coalescing on release.
class Arena {
  public:
    size_t cap = 0, used = 0, peak = 0;
    void init(size_t c) {
        cap = c & ~(size_t)255;
        free_.clear();
        free_[0] = cap;
        used = peak = 0;
    }
    bool alloc(size_t n, size_t* off) {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n;
            const size_t at = it->first + n;
            free_.erase(it);
            if (rest) free_[at] = rest;
            used += n;
            peak = std::max(peak, used);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) & ~(size_t)255;
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

struct Request {
    long long id = 0;
    bool large = false;
    acs_settings set{};        // the server's settings with this request's overrides
    double tol = 1e-6;
    int max_iter = 0;
    // host copy of the problem (needed again only by the whole-GPU path)
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col, dims;
    std::vector<double> val, b, c;
    int n_orth = 0;
    // pool layout: offsets relative to the request's block
    Matrix X;
    Member M;
    double* dM = nullptr;
    double* dX = nullptr;
    std::vector<char> image;   // the static part (matrix, b, c, cone offsets)
    size_t static_bytes = 0, bytes = 0, off = 0;
    int slot = -1;
    bool started = false;
    // results
    bool done = false;
    int status = ACS_ERR_CUDA, iters = 0;
    double res[8] = {0};
    std::vector<double> x, y, s;
    Clock::time_point t_submit, t_done;
};

}  // namespace

struct Server {
    acs_settings set{};
    acs_server_config cfg{};
    int device = 0, nsm = 0;
    cudaStream_t stream = nullptr;
    char* arena_base = nullptr;
    Arena arena;
    acs_batch_mapping map{256, 1};
    int grid = 0, max_ctas = 0, slots = 0;
    // slot arrays
    IterParams<float>* d_p32 = nullptr;
    IterParams<double>* d_p64 = nullptr;
    Control* d_ctl = nullptr;
    int* d_order = nullptr;
    int* d_head = nullptr;
    int* d_mailbox = nullptr;
    unsigned long long* d_team_bar = nullptr;
    double* d_team_part = nullptr;
    int* d_team_err = nullptr;
    int* d_cta = nullptr;                         // [3 * max_ctas] assigned teams: k, rank, size
    unsigned long long* d_t0 = nullptr;
    int* d_cond_list = nullptr;
    std::vector<int> cond_list_host;
    std::vector<void*> allocations;
    std::vector<int> free_slots;
    std::vector<Control> ctl_host;
    // queue
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Request*> pending;
    std::vector<Request*> active;                 // worker only
    std::unordered_map<long long, Request*> reqs;
    long long next_id = 1;
    bool stop = false;
    std::thread worker;
    // statistics
    long long n_rounds = 0, n_admitted = 0, n_done = 0, n_large = 0;
    double round_ms_sum = 0.0, active_sum = 0.0;
    double short_credit_ms = 0.0;                 // round time the short class is owed
};

namespace {

template <typename T>
int salloc(Server* S, T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return ACS_ERR_OOM;
    }
    S->allocations.push_back(q);
    *p = static_cast<T*>(q);
    return ACS_SOLVED;
}

// Layout of one request inside its pool block (dry run from offset 0).
void request_layout(Request* R, Pool& P) {
    Matrix& X = R->X;
    Member& M = R->M;
    const bool bf16 = R->set.a_storage == ACS_STORE_BF16;
    layout_sell(P, X.H.A, X.dA, bf16);
    layout_sell(P, X.H.AT, X.dAT, bf16);
    M.db = P.take<double>(M.m);
    M.dc = P.take<double>(M.n);
    M.dsoc = P.take<int>(M.n_soc + 1);
    R->static_bytes = P.off;
    const int m = M.m, n = M.n;
    M.x = P.take<double>(n);
    M.z = P.take<double>(n);
    M.ocone = P.take<double>((size_t)M.n_orth + M.n_soc);
    Outer& O = M.X;
    O.s = P.take<double>(n); O.p = P.take<double>(n); O.g = P.take<double>(n);
    O.q = P.take<double>(n); O.chat = P.take<double>(n); O.O = P.take<double>(n);
    O.w = P.take<double>(m); O.btil = P.take<double>(m);
    O.wp = P.take<double>(m); O.qp = P.take<double>(n);
    auto inner = [&](auto& V) {
        using T = std::remove_pointer_t<decltype(V.r)>;
        V.r = P.take<T>(m); V.u = P.take<T>(m); V.p = P.take<T>(m); V.sv = P.take<T>(m);
        V.au = P.take<T>(m); V.jinv = P.take<T>(m); V.t = P.take<T>(n); V.O2 = P.take<T>(n);
    };
    inner(M.V32);
    inner(M.V64);
    if (M.dense) {
        R->dM = P.take<double>((size_t)m * m);
        R->dX = P.take<double>((size_t)m * m);
    }
    R->bytes = P.off;
}

// Host image of the static part of the block.
void request_image(Request* R) {
    R->image.assign(R->static_bytes, 0);
    image_sell(R->image, R->X.H.A, R->X.dA);
    image_sell(R->image, R->X.H.AT, R->X.dAT);
    put_bytes(R->image.data(), R->M.db, R->M.b.data(), R->M.b.size());
    put_bytes(R->image.data(), R->M.dc, R->M.c.data(), R->M.c.size());
    put_bytes(R->image.data(), R->M.dsoc, R->M.soc_off.data(), R->M.soc_off.size());
}

Control fresh_control(double eta0) {
    Control c;
    memset(&c, 0, sizeof(c));
    c.status = ST_RUNNING;
    for (int k = 0; k < 6; ++k) c.res[k] = NAN;
    c.ds = INFINITY;
    c.eta = eta0;
    return c;
}

cudaError_t write_params(Server* S, Request* R) {
    const int ncl = (int)S->cond_list_host.size();
    const Member& M = R->M;
    IterParams<float> p32 = member_params<float>(R->set, S->d_cond_list, ncl, M, R->X, M.V32, R->tol, R->max_iter);
    IterParams<double> p64 = member_params<double>(R->set, S->d_cond_list, ncl, M, R->X, M.V64, R->tol, R->max_iter);
    p32.ctl = p64.ctl = S->d_ctl + R->slot;
    p32.refresh = p64.refresh = R->started ? 1 : 0;
    p64.dM = R->dM;
    p64.dX = R->dX;
    p64.own_scratch = R->dM ? 1 : 0;
    cudaError_t e = cudaMemcpyAsync(S->d_p32 + R->slot, &p32, sizeof(p32), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->d_p64 + R->slot, &p64, sizeof(p64), cudaMemcpyHostToDevice, S->stream);
    return e;
}

// Upload an admitted request into its block and slot (worker thread).
// Returns the first CUDA error of the uploads (the caller then retires the
// request with ACS_ERR_CUDA instead of running it).
cudaError_t admit(Server* S, Request* R) {
    char* base = S->arena_base + R->off;
    cudaError_t e = cudaMemcpyAsync(base, R->image.data(), R->static_bytes, cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + R->static_bytes, 0, R->bytes - R->static_bytes, S->stream);
    std::vector<char>().swap(R->image);
    // offsets -> device addresses
    // (the shapes were recorded at submission, when the host image was built)
    rebase_sell(R->X.dA, base, R->X.A);
    rebase_sell(R->X.dAT, base, R->X.AT);
    Member& M = R->M;
    M.db = rebase(M.db, base); M.dc = rebase(M.dc, base); M.dsoc = rebase(M.dsoc, base);
    M.x = rebase(M.x, base); M.z = rebase(M.z, base); M.ocone = rebase(M.ocone, base);
    Outer& O = M.X;
    O.s = rebase(O.s, base); O.p = rebase(O.p, base); O.g = rebase(O.g, base); O.q = rebase(O.q, base);
    O.chat = rebase(O.chat, base); O.O = rebase(O.O, base); O.w = rebase(O.w, base); O.btil = rebase(O.btil, base);
    O.wp = rebase(O.wp, base); O.qp = rebase(O.qp, base);
    auto inner = [&](auto& V) {
        V.r = rebase(V.r, base); V.u = rebase(V.u, base); V.p = rebase(V.p, base); V.sv = rebase(V.sv, base);
        V.au = rebase(V.au, base); V.jinv = rebase(V.jinv, base); V.t = rebase(V.t, base); V.O2 = rebase(V.O2, base);
    };
    inner(M.V32);
    inner(M.V64);
    if (R->dM) {
        R->dM = rebase(R->dM, base);
        R->dX = rebase(R->dX, base);
    }
    const Control c = fresh_control(S->set.cg_eta);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_ctl + R->slot, &c, sizeof(c), cudaMemcpyHostToDevice, S->stream);
    R->started = false;
    if (e == cudaSuccess) e = write_params(S, R);
    return e;
}

void finish(Server* S, Request* R) {
    R->t_done = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    R->done = true;
    ++S->n_done;
    S->cv_done.notify_all();
}

// Copy a finished request's results out and release its block and slot.
void retire(Server* S, Request* R, const Control& C) {
    const Member& M = R->M;
    R->x.resize(M.n);
    R->s.resize(M.n);
    std::vector<double> w(M.m);
    // a copy that fails leaves the host results undefined: the request then
    // reports the CUDA error instead of its device-side status
    cudaError_t e = cudaMemcpyAsync(R->x.data(), M.x, sizeof(double) * M.n, cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R->s.data(), M.z, sizeof(double) * M.n, cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.data(), M.X.w, sizeof(double) * M.m, cudaMemcpyDeviceToHost, S->stream);
    const cudaError_t es = cudaStreamSynchronize(S->stream);
    if (e == cudaSuccess) e = es;
    R->y.resize(M.m);
    for (int r = 0; r < M.m; ++r) R->y[R->X.H.perm[r]] = w[r] / S->set.mu;
    R->status = e == cudaSuccess ? member_status(C) : ACS_ERR_CUDA;
    R->iters = C.l;
    for (int k = 0; k < 6; ++k) R->res[k] = C.res[k];
    R->res[6] = (double)C.cg_iters;
    R->res[7] = (double)C.switched_at;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->arena.release(R->off, R->bytes);
        S->free_slots.push_back(R->slot);
    }
    R->slot = -1;
    finish(S, R);
}

// A large request: alone on the whole GPU through the single-problem launch.
void run_large(Server* S, Request* R) {
    acs_settings st = R->set;
    st.cuda_stream = S->stream;
    st.cond_list = S->cond_list_host.empty() ? nullptr : S->cond_list_host.data();
    st.n_cond_list = (int32_t)S->cond_list_host.size();
    acs_problem* h = nullptr;
    const int m = (int)R->b.size(), n = (int)R->c.size();
    int rc = acs_problem_create(m, n, R->row_ptr.data(), R->col.data(), R->val.data(), R->b.data(), R->c.data(),
                                R->n_orth, (int32_t)R->dims.size(), R->dims.empty() ? nullptr : R->dims.data(), &st, &h);
    if (rc == ACS_SOLVED) rc = acs_solve(h, R->tol, R->max_iter);
    if (h) {
        R->x.resize(n);
        R->y.resize(m);
        R->s.resize(n);
        int32_t it = 0;
        const int g = acs_get(h, R->x.data(), R->y.data(), R->s.data(), &it, R->res);
        R->iters = it;
        rc = g;
        acs_problem_destroy(h);
    }
    R->status = rc;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->n_large;
    }
    finish(S, R);
}

int pow2_floor(long long v) {
    int p = 1;
    while ((long long)p * 2 <= v) p *= 2;
    return p;
}

// Teams of their own for the requests of a round with fewer requests than
// CTAs: every request gets a power-of-two team sized by its share of the
// round's work (stored entries, vectors, and m^2 for a cached dense factor),
// capped where more CTAs would only add barrier cost (one CTA per 16384
// units of work); spare CTAs go to the requests with the most work per CTA.
// Fills cta[3 * grid] = (position in order or -1, rank, team size).
double team_work(const Member& M) {
    return (double)M.nnz * 2 + M.m + M.n + (M.dense ? 0.25 * (double)M.m * M.m : 0.0);
}

// w[k]: work of request k; requires 1 <= w.size() <= grid.
void assign_teams_w(const std::vector<double>& w, int grid, std::vector<int>& cta) {
    const int n = (int)w.size();
    std::vector<int> g(n), cap(n);
    double total = 0.0;
    for (int k = 0; k < n; ++k) {
        total += w[k];
        cap[k] = std::min(pow2_floor(std::max(1LL, (long long)(w[k] / 16384.0))), std::min(grid, kMaxGrid));
    }
    long long used = 0;
    for (int k = 0; k < n; ++k) {
        g[k] = std::min(cap[k], pow2_floor(std::max(1LL, (long long)(grid * w[k] / total))));
        used += g[k];
    }
    while (used > grid) {                          // halve the largest team
        int j = (int)(std::max_element(g.begin(), g.end()) - g.begin());
        if (g[j] == 1) break;                      // (cannot happen while n <= grid)
        used -= g[j] / 2;
        g[j] /= 2;
    }
    while (true) {                                 // double where work per CTA is largest
        int best = -1;
        for (int k = 0; k < n; ++k)
            if (g[k] < cap[k] && used + g[k] <= grid && (best < 0 || w[k] / g[k] > w[best] / g[best])) best = k;
        if (best < 0) break;
        used += g[best];
        g[best] *= 2;
    }
    cta.assign(3 * (size_t)grid, 0);
    for (int b = 0; b < grid; ++b) cta[b] = -1;
    int b = 0;
    for (int k = 0; k < n; ++k)
        for (int r = 0; r < g[k]; ++r, ++b) {
            cta[b] = k;
            cta[grid + b] = r;
            cta[2 * grid + b] = g[k];
        }
}

void assign_teams(const std::vector<Request*>& act, int grid, std::vector<int>& cta) {
    std::vector<double> w(act.size());
    for (size_t k = 0; k < act.size(); ++k) w[k] = team_work(act[k]->M);
    assign_teams_w(w, grid, cta);
}

bool is_long(const Server* S, const Request* R) {
    return S->cfg.long_nnz > 0 && R->M.nnz > S->cfg.long_nnz;
}

// One time-sliced launch over the active requests of a class (-1: all, 0:
// short, 1: long); retire the finished.  Returns the round's wall time (ms).
double run_round(Server* S, int cls) {
    std::vector<Request*> act, others;
    for (Request* R : S->active) {
        if (cls < 0 || (int)is_long(S, R) == cls) act.push_back(R);
        else others.push_back(R);
    }
    std::sort(act.begin(), act.end(), [](const Request* a, const Request* b) { return a->id < b->id; });
    std::vector<int> order(act.size());
    for (size_t k = 0; k < act.size(); ++k) order[k] = act[k]->slot;
    cudaStream_t st = S->stream;
    cudaMemcpyAsync(S->d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, st);
    // fewer requests than CTAs: teams of their own, sized by work
    const bool assigned = S->cfg.adaptive_teams != 0 && (int)act.size() <= S->grid;
    std::vector<int> cta;
    if (assigned) {
        assign_teams(act, S->grid, cta);
        cudaMemcpyAsync(S->d_cta, cta.data(), sizeof(int) * cta.size(), cudaMemcpyHostToDevice, st);
    }
    cudaMemsetAsync(S->d_head, 0, sizeof(int), st);
    cudaMemsetAsync(S->d_t0, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(S->d_team_bar, 0, sizeof(unsigned long long) * S->max_ctas, st);
    cudaMemsetAsync(S->d_team_err, 0, sizeof(int) * S->max_ctas, st);
    BatchArgs a{};
    a.count = (int)order.size();
    a.order = S->d_order;
    a.p32 = S->d_p32;
    a.p64 = S->d_p64;
    a.ctl = S->d_ctl;
    a.head = S->d_head;
    a.mailbox = S->d_mailbox;
    a.team_bar = S->d_team_bar;
    a.team_part = S->d_team_part;
    a.team_err = S->d_team_err;
    a.dense = nullptr;                            // requests keep their own scratch
    a.dense_m2 = 0;
    a.round_t0 = S->d_t0;
    a.round_ns = (unsigned long long)(S->cfg.round_ms * 1e6);
    a.g = S->map.team_ctas;
    a.fp64 = S->set.precision == ACS_PREC_FP64 ? 1 : 0;
    if (assigned) {
        a.cta_k = S->d_cta;
        a.cta_rank = S->d_cta + S->grid;
        a.cta_g = S->d_cta + 2 * S->grid;
    }
    void* args[] = {(void*)&a};
    const auto t0 = Clock::now();
    cudaError_t e = cudaLaunchCooperativeKernel(kernel_for(S->map.threads_per_cta), dim3(S->grid),
                                                dim3(S->map.threads_per_cta), args, 0, st);
    S->ctl_host.resize(S->slots);
    const int top = 1 + *std::max_element(order.begin(), order.end());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->ctl_host.data(), S->d_ctl, sizeof(Control) * top, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->n_rounds;
        S->round_ms_sum += ms;
        S->active_sum += (double)act.size();
    }
    std::vector<Request*> keep;
    for (Request* R : act) {
        const Control& C = S->ctl_host[R->slot];
        if (e != cudaSuccess) {
            Control bad = fresh_control(0.0);
            bad.status = ACS_ERR_CUDA;
            retire(S, R, bad);
            continue;
        }
        const int s = C.status;
        if (s == ST_PAUSED || s == ST_RUNNING || s == ST_SWITCH) {
            if (!R->started && C.l > 0) {
                R->started = true;
                write_params(S, R);                    // from now on it resumes
            }
            keep.push_back(R);
        } else {
            retire(S, R, C);
        }
    }
    others.insert(others.end(), keep.begin(), keep.end());
    S->active.swap(others);
    if (e != cudaSuccess) fprintf(stderr, "acs: serving round failed: %s\n", cudaGetErrorString(e));
    return ms;
}

void worker_main(Server* S) {
    cudaSetDevice(S->device);
    while (true) {
        std::vector<Request*> admitted;
        Request* large = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
            if (S->stop && S->pending.empty() && S->active.empty()) break;
            while (!S->pending.empty()) {
                Request* R = S->pending.front();
                if (R->large) {
                    large = R;
                    S->pending.pop_front();
                    break;
                }
                if (S->free_slots.empty()) break;
                size_t off = 0;
                if (!S->arena.alloc(R->bytes, &off)) break;   // waits for memory to free up
                R->off = off;
                R->slot = S->free_slots.back();
                S->free_slots.pop_back();
                S->pending.pop_front();
                admitted.push_back(R);
                ++S->n_admitted;
            }
        }
        for (Request* R : admitted) {
            if (admit(S, R) == cudaSuccess) {
                S->active.push_back(R);
            } else {
                cudaGetLastError();
                Control bad = fresh_control(0.0);
                bad.status = ACS_ERR_CUDA;
                retire(S, R, bad);
            }
        }
        if (large) run_large(S, large);
        if (!S->active.empty()) {
            // with both classes admitted, alternate with equal time for each:
            // a long request's iteration can outlast the deadline by far, and
            // short requests would wait idle for it in a shared round
            int n_long = 0;
            for (const Request* R : S->active) n_long += is_long(S, R) ? 1 : 0;
            const int n_short = (int)S->active.size() - n_long;
            if (n_long == 0 || n_short == 0) {
                run_round(S, -1);
                S->short_credit_ms = 0.0;
            } else if (S->short_credit_ms > 0.0) {
                S->short_credit_ms -= run_round(S, 0);
            } else {
                S->short_credit_ms += run_round(S, 1);
            }
        }
    }
}

}  // namespace
}  // namespace acs

using acs::Server;

extern "C" {

int acs_server_config_default(acs_server_config* c) {
    if (!c) return ACS_ERR_ARG;
    c->budget_bytes = (int64_t)4 << 30;
    c->max_active = 2048;
    c->round_ms = 2.0;
    c->large_nnz = (int64_t)1 << 23;
    c->threads_per_cta = 256;
    c->team_ctas = 1;
    c->long_nnz = 262144;
    c->adaptive_teams = 1;
    return ACS_SOLVED;
}

int acs_server_create(const acs_settings* settings, const acs_server_config* cfg, acs_server** out) {
    using namespace acs;
    if (!out) return ACS_ERR_ARG;
    *out = nullptr;
    acs_settings set;
    if (settings) set = *settings; else acs_settings_default(&set);
    if (!host::valid_settings(set)) return ACS_ERR_ARG;
    acs_server_config c;
    if (cfg) c = *cfg; else acs_server_config_default(&c);
    const acs_batch_mapping map{c.threads_per_cta, c.team_ctas};
    if (c.budget_bytes < (1 << 20) || c.max_active <= 0 || !(c.round_ms > 0) || c.large_nnz < 0 || c.long_nnz < 0 ||
        !valid_mapping(map))
        return ACS_ERR_ARG;
    Server* S = new (std::nothrow) Server();
    if (!S) return ACS_ERR_OOM;
    S->set = set;
    S->cfg = c;
    S->map = map;
    S->device = set.device;
    if (set.n_cond_list > 0) S->cond_list_host.assign(set.cond_list, set.cond_list + set.n_cond_list);
    S->set.cond_list = nullptr;
    S->set.cuda_stream = nullptr;
    auto fail = [&](int rc) {
        for (void* p : S->allocations) cudaFree(p);
        if (S->stream) cudaStreamDestroy(S->stream);
        delete S;
        return rc;
    };
    if (cudaSetDevice(S->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(ACS_ERR_CUDA);
    int bps = 0;
    if (occupancy_for(map.threads_per_cta, &bps) != ACS_SOLVED) return fail(ACS_ERR_CUDA);
    S->grid = S->nsm * bps;
    S->grid -= S->grid % map.team_ctas;
    S->max_ctas = S->grid;
    S->slots = c.max_active;
    if (cudaMalloc(&S->arena_base, (size_t)c.budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ACS_ERR_OOM);
    }
    S->allocations.push_back(S->arena_base);
    S->arena.init((size_t)c.budget_bytes);
    int rc = 0;
    rc |= salloc(S, &S->d_p32, S->slots);
    rc |= salloc(S, &S->d_p64, S->slots);
    rc |= salloc(S, &S->d_ctl, S->slots);
    rc |= salloc(S, &S->d_order, S->slots);
    rc |= salloc(S, &S->d_head, 1);
    rc |= salloc(S, &S->d_mailbox, S->max_ctas);
    rc |= salloc(S, &S->d_team_bar, S->max_ctas);
    rc |= salloc(S, &S->d_team_part, (size_t)S->max_ctas * kMaxRed);
    rc |= salloc(S, &S->d_team_err, S->max_ctas);
    rc |= salloc(S, &S->d_cta, 3 * (size_t)S->max_ctas);
    rc |= salloc(S, &S->d_t0, 1);
    rc |= salloc(S, &S->d_cond_list, S->cond_list_host.size());
    if (rc) return fail(ACS_ERR_OOM);
    if (!S->cond_list_host.empty() &&
        cudaMemcpy(S->d_cond_list, S->cond_list_host.data(), sizeof(int) * S->cond_list_host.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ACS_ERR_CUDA);
    S->free_slots.resize(S->slots);
    for (int i = 0; i < S->slots; ++i) S->free_slots[i] = S->slots - 1 - i;
    S->worker = std::thread(acs::worker_main, S);
    *out = reinterpret_cast<acs_server*>(S);
    return ACS_SOLVED;
}

int acs_server_submit(acs_server* h, const acs_instance* I, double tol, int32_t max_iter,
                      const acs_settings* per_request, int64_t* id) {
    using namespace acs;
    Server* S = reinterpret_cast<Server*>(h);
    if (!S || !I || !id || !(tol >= 0) || max_iter < 0 || I->share_A_with != -1) return ACS_ERR_ARG;
    acs_settings rs = S->set;
    if (per_request) {
        if (per_request->n_cond_list != 0) return ACS_ERR_ARG;
        rs.mu = per_request->mu;
        rs.t = per_request->t;
        rs.cond_first = per_request->cond_first;
        rs.cond_period = per_request->cond_period;
        rs.check_every = per_request->check_every;
        if (!host::valid_settings(rs)) return ACS_ERR_ARG;
    }
    const int vrc = host::no_throw([&] {
        return host::validate(I->m, I->n, I->row_ptr, I->col, I->val, I->b, I->c, I->n_orthant, I->n_soc,
                              I->soc_dims);
    });
    if (vrc != ACS_SOLVED) return vrc;
    const Clock::time_point t_entry = Clock::now();   // latency includes the host preparation
    Request* R = new (std::nothrow) Request();
    if (!R) return ACS_ERR_OOM;
    const int prc = host::no_throw([&]() -> int {
        R->tol = tol;
        R->max_iter = max_iter;
        R->set = rs;
        const long long nnz = I->row_ptr[I->m];
        R->large = nnz > S->cfg.large_nnz;
        if (R->large) {
            R->row_ptr.assign(I->row_ptr, I->row_ptr + I->m + 1);
            R->col.assign(I->col, I->col + nnz);
            R->val.assign(I->val, I->val + nnz);
            R->b.assign(I->b, I->b + I->m);
            R->c.assign(I->c, I->c + I->n);
            R->dims.assign(I->soc_dims, I->soc_dims + I->n_soc);
            R->n_orth = I->n_orthant;
        } else {
            // the same preparation as a batch member (lanes per row for one CTA)
            if (host::build(I->m, I->n, I->row_ptr, I->col, I->val, I->b, I->c, I->n_orthant, I->n_soc, I->soc_dims,
                            (long long)S->map.threads_per_cta / 32, (long long)S->map.threads_per_cta / 32,
                            R->X.H) != ACS_SOLVED)
                return ACS_ERR_CSR;
            R->X.stored = (long long)R->X.H.A.col.size();
            Member& M = R->M;
            M.m = I->m; M.n = I->n; M.n_orth = I->n_orthant; M.n_soc = I->n_soc; M.mat = 0;
            M.dense = host::dense_mode(rs, I->m);
            M.nnz = R->X.stored;
            M.b = R->X.H.bperm;
            M.c.assign(I->c, I->c + I->n);
            M.soc_off = R->X.H.soc_off;
            M.bnorm = R->X.H.bnorm;
            M.cnorm = R->X.H.cnorm;
            Pool dry;
            request_layout(R, dry);
            if (R->bytes + 4096 > S->arena.cap) return ACS_ERR_LIMIT;
            request_image(R);
            auto shape = [](const host::HostSell& H, SellMat& Sm) {
                Sm.nrows = H.nrows; Sm.nslices = H.nslices; Sm.g = H.g;
            };
            shape(R->X.H.A, R->X.A);
            shape(R->X.H.AT, R->X.AT);
            // the host images are no longer needed (keep the row relabelling)
            std::vector<int> perm = std::move(R->X.H.perm);
            R->X.H = host::HostProblem();
            R->X.H.perm = std::move(perm);
            std::vector<double>().swap(M.b);
            std::vector<double>().swap(M.c);
        }
        return ACS_SOLVED;
    });
    if (prc != ACS_SOLVED) {
        delete R;
        return prc;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        R->id = S->next_id++;
        R->t_submit = t_entry;
        try {
            S->reqs[R->id] = R;
            S->pending.push_back(R);
        } catch (...) {                                  // host memory: undo the registration
            S->reqs.erase(R->id);
            delete R;
            return ACS_ERR_OOM;
        }
        *id = R->id;
    }
    S->cv.notify_one();
    return ACS_SOLVED;
}

int acs_server_poll(acs_server* h, int64_t id, int32_t* done) {
    Server* S = reinterpret_cast<Server*>(h);
    if (!S || !done) return ACS_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return ACS_ERR_ARG;
    *done = it->second->done ? 1 : 0;
    return ACS_SOLVED;
}

int acs_server_wait(acs_server* h, int64_t id, double timeout_s) {
    Server* S = reinterpret_cast<Server*>(h);
    if (!S) return ACS_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->reqs.find(id) == S->reqs.end()) return ACS_ERR_ARG;
    // look the request up again on every wake-up: another thread's
    // acs_server_result may have taken (and freed) it meanwhile
    auto ready = [&] {
        auto it = S->reqs.find(id);
        return it == S->reqs.end() || it->second->done;
    };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return ACS_ERR_DEVICE_TIMEOUT;
    }
    auto it = S->reqs.find(id);
    return it == S->reqs.end() ? ACS_ERR_ARG : it->second->status;
}

int acs_server_result(acs_server* h, int64_t id, double* x, double* y, double* sl, int32_t* iters, double* residuals,
                      double* latency_ms) {
    Server* S = reinterpret_cast<Server*>(h);
    if (!S) return ACS_ERR_ARG;
    acs::Request* R = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end() || !it->second->done) return ACS_ERR_ARG;
        R = it->second;
        S->reqs.erase(it);
    }
    if (x) std::copy(R->x.begin(), R->x.end(), x);
    if (y) std::copy(R->y.begin(), R->y.end(), y);
    if (sl) std::copy(R->s.begin(), R->s.end(), sl);
    if (iters) *iters = R->iters;
    if (residuals) std::copy(R->res, R->res + 8, residuals);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(R->t_done - R->t_submit).count();
    const int st = R->status;
    delete R;
    return st;
}

int acs_server_stats(acs_server* h, double* out) {
    Server* S = reinterpret_cast<Server*>(h);
    if (!S || !out) return ACS_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    out[0] = (double)S->n_rounds;
    out[1] = (double)S->n_admitted;
    out[2] = (double)S->n_done;
    out[3] = (double)(S->n_admitted - (S->n_done - S->n_large));
    out[4] = (double)S->arena.used;
    out[5] = (double)S->arena.peak;
    out[6] = (double)S->n_large;
    out[7] = (double)S->pending.size();
    out[8] = S->n_rounds ? S->round_ms_sum / S->n_rounds : 0.0;
    out[9] = S->n_rounds ? S->active_sum / S->n_rounds : 0.0;
    return ACS_SOLVED;
}

int acs_debug_assign_teams(int32_t n, const double* work, int32_t grid, int32_t* cta) {
    if (n <= 0 || grid <= 0 || n > grid || !work || !cta) return ACS_ERR_ARG;
    return acs::host::no_throw([&]() -> int {
        std::vector<double> w(work, work + n);
        for (double v : w)
            if (!(v > 0)) return ACS_ERR_ARG;
        std::vector<int> c;
        acs::assign_teams_w(w, grid, c);
        std::copy(c.begin(), c.end(), cta);
        return ACS_SOLVED;
    });
}

int acs_debug_arena(int64_t cap, int32_t nops, const int64_t* ops, int64_t* offsets, int64_t* used_peak) {
    if (cap <= 0 || nops < 0 || (nops > 0 && (!ops || !offsets)) || !used_peak) return ACS_ERR_ARG;
    return acs::host::no_throw([&]() -> int {
        acs::Arena A;
        A.init((size_t)cap);
        std::vector<int64_t> size_of(nops, 0);
        for (int k = 0; k < nops; ++k) {
            if (ops[k] > 0) {
                size_t off = 0;
                offsets[k] = A.alloc((size_t)ops[k], &off) ? (int64_t)off : -1;
                size_of[k] = offsets[k] >= 0 ? ops[k] : 0;
            } else {
                const int64_t j = -ops[k] - 1;              // free the block of op j
                if (j < 0 || j >= k || ops[j] <= 0 || offsets[j] < 0 || size_of[j] == 0) return ACS_ERR_ARG;
                A.release((size_t)offsets[j], (size_t)size_of[j]);
                size_of[j] = 0;
                offsets[k] = -1;
            }
        }
        used_peak[0] = (int64_t)A.used;
        used_peak[1] = (int64_t)A.peak;
        return ACS_SOLVED;
    });
}

void acs_server_destroy(acs_server* h) {
    Server* S = reinterpret_cast<Server*>(h);
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->device);
    for (auto& kv : S->reqs) delete kv.second;
    for (void* p : S->allocations) cudaFree(p);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
}

}  // extern "C"
