// Batched solves: many independent conic programs of uneven sizes in one
// persistent launch, replayed from a captured CUDA graph.
//
// Device design.  The launch is one cooperative grid of resident CTAs split
// into fixed teams of g consecutive CTAs (g = 1 for most batches).  A team's
// rank-0 CTA takes the next member from a global counter (members ordered by
// decreasing size, so the longest solves start first and the tail is short),
// posts it to the team, and the team runs that member's whole solve --
// Algorithm 2 (arXiv 2103.00736, Section IV) with the same phases as the
// single-problem kernel -- synchronising only among its own CTAs (a team of
// one CTA needs no global barrier at all).  Then it takes the next member.
// The mixed-precision hand-over (FP32 correction solve -> FP64) happens inside
// the same launch.  Members sharing one A point at a single device copy of it,
// so their matrix passes hit in L2.
//
// Host design.  Every member is prepared like a single problem (validation,
// relabelled rows, sliced-ELLPACK A and A'), then all device data live in one
// allocation: a static region (matrices, b, c, cone offsets) uploaded once
// from a host image, and a state region (iterates, solver vectors) zeroed once.

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <atomic>
#include <numeric>
#include <vector>

#include "acs_team.cuh"

namespace acs {

struct Batch {
    int count = 0, device = 0, nsm = 0;
    acs_settings set{};
    std::vector<int> cond_list_host;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<Matrix> mats;
    std::vector<Member> mem;
    std::vector<int> order;
    // pool
    char* pool = nullptr;
    size_t static_bytes = 0, total_bytes = 0;
    int* d_cond_list = nullptr;
    int* d_order = nullptr;
    IterParams<float>* d_p32 = nullptr;
    IterParams<double>* d_p64 = nullptr;
    Control* d_ctl = nullptr;
    int* d_head = nullptr;
    int* d_mailbox = nullptr;
    unsigned long long* d_team_bar = nullptr;
    double* d_team_part = nullptr;
    int* d_team_err = nullptr;
    double* d_dense = nullptr;
    long long dense_m2 = 0;
    int max_ctas = 0;
    // mapping and launch
    acs_batch_mapping map{1024, 1};
    int grid = 0;
    double p_tol = -1.0;
    int p_max_iter = -1;
    cudaGraphExec_t gexec = nullptr;
    bool graph_ok = false, last_graph = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    std::vector<Control> ctl_host;
};

namespace {

// CTAs of a launch under mapping m: every resident CTA, in whole teams.
int grid_for(Batch* B, const acs_batch_mapping& m, int* grid) {
    int bps = 0;
    if (occupancy_for(m.threads_per_cta, &bps) != ACS_SOLVED) return ACS_ERR_CUDA;
    int g = B->nsm * bps;
    g -= g % m.team_ctas;
    if (g < m.team_ctas || g > B->max_ctas) return ACS_ERR_ARG;
    *grid = g;
    return ACS_SOLVED;
}

// Write the per-member parameter blocks for (tol, max_iter).
int upload_params(Batch* B, double tol, int max_iter) {
    std::vector<IterParams<float>> p32(B->count);
    std::vector<IterParams<double>> p64(B->count);
    for (int i = 0; i < B->count; ++i) {
        const Member& M = B->mem[i];
        const int ncl = (int)B->cond_list_host.size();
        p32[i] = member_params<float>(B->set, B->d_cond_list, ncl, M, B->mats[M.mat], M.V32, tol, max_iter);
        p64[i] = member_params<double>(B->set, B->d_cond_list, ncl, M, B->mats[M.mat], M.V64, tol, max_iter);
        p32[i].ctl = B->d_ctl + i;
        p64[i].ctl = B->d_ctl + i;
    }
    if (cudaMemcpyAsync(B->d_p32, p32.data(), sizeof(p32[0]) * B->count, cudaMemcpyHostToDevice, B->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(B->d_p64, p64.data(), sizeof(p64[0]) * B->count, cudaMemcpyHostToDevice, B->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    B->p_tol = tol;
    B->p_max_iter = max_iter;
    return ACS_SOLVED;
}

BatchArgs batch_args(Batch* B) {
    BatchArgs a{};
    a.count = B->count;
    a.order = B->d_order;
    a.p32 = B->d_p32;
    a.p64 = B->d_p64;
    a.ctl = B->d_ctl;
    a.head = B->d_head;
    a.mailbox = B->d_mailbox;
    a.team_bar = B->d_team_bar;
    a.team_part = B->d_team_part;
    a.team_err = B->d_team_err;
    a.dense = B->dense_m2 > 0 ? B->d_dense : nullptr;
    a.dense_m2 = B->dense_m2;
    a.g = B->map.team_ctas;
    a.fp64 = B->set.precision == ACS_PREC_FP64 ? 1 : 0;
    return a;
}

// Reset + persistent launch on the batch's stream (captured or direct).
cudaError_t enqueue(Batch* B) {
    BatchArgs a = batch_args(B);
    const int teams = B->grid / B->map.team_ctas;
    batch_reset<<<(B->count + 255) / 256, 256, 0, B->stream>>>(a, B->set.cg_eta);
    batch_reset_teams<<<(teams + 255) / 256, 256, 0, B->stream>>>(a, teams);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel(kernel_for(B->map.threads_per_cta), dim3(B->grid),
                                       dim3(B->map.threads_per_cta), args, 0, B->stream);
}

void drop_graph(Batch* B) {
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
    B->graph_ok = false;
}

int set_mapping(Batch* B, const acs_batch_mapping& m) {
    if (!valid_mapping(m)) return ACS_ERR_ARG;
    int grid = 0;
    const int rc = grid_for(B, m, &grid);
    if (rc != ACS_SOLVED) return rc;
    if (m.threads_per_cta != B->map.threads_per_cta || m.team_ctas != B->map.team_ctas) drop_graph(B);
    B->map = m;
    B->grid = grid;
    return ACS_SOLVED;
}

int launch(Batch* B, double tol, int max_iter, bool use_graph) {
    if (tol != B->p_tol || max_iter != B->p_max_iter) {
        drop_graph(B);
        const int rc = upload_params(B, tol, max_iter);
        if (rc != ACS_SOLVED) return rc;
    }
    cudaStream_t st = B->stream;
    if (use_graph && !B->gexec) {
        // capture once; if capturing the cooperative launch is refused, the
        // work is launched directly instead (reported by acs_batch_info)
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t e1 = enqueue(B);
            const cudaError_t e2 = cudaStreamEndCapture(st, &g);
            if (e1 == cudaSuccess && e2 == cudaSuccess && g &&
                cudaGraphInstantiate(&B->gexec, g, 0) == cudaSuccess) {
                B->graph_ok = true;
            } else {
                B->gexec = nullptr;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    cudaEventRecord(B->ev[0], st);
    cudaError_t e;
    if (use_graph && B->gexec) {
        e = cudaGraphLaunch(B->gexec, st);
        B->last_graph = true;
    } else {
        e = enqueue(B);
        B->last_graph = false;
    }
    cudaEventRecord(B->ev[1], st);
    if (e != cudaSuccess) {
        fprintf(stderr, "acs: batched launch failed: %s\n", cudaGetErrorString(e));
        return ACS_ERR_CUDA;
    }
    return ACS_SOLVED;
}

int fetch_controls(Batch* B) {
    B->ctl_host.resize(B->count);
    if (cudaMemcpyAsync(B->ctl_host.data(), B->d_ctl, sizeof(Control) * B->count, cudaMemcpyDeviceToHost,
                        B->stream) != cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess)
        return ACS_ERR_CUDA;
    return ACS_SOLVED;
}

// Lay out (dry run with base = 0, then for real) every device buffer.
void layout(Batch* B, Pool& P) {
    const int count = B->count;
    // static region: matrices, then per-member b, c, cone offsets, cond list
    for (Matrix& X : B->mats) {
        const bool bf16 = B->set.a_storage == ACS_STORE_BF16;
        layout_sell(P, X.H.A, X.dA, bf16);
        layout_sell(P, X.H.AT, X.dAT, bf16);
    }
    for (Member& M : B->mem) {
        M.db = P.take<double>(M.m);
        M.dc = P.take<double>(M.n);
        M.dsoc = P.take<int>(M.n_soc + 1);
    }
    B->d_cond_list = P.take<int>(B->cond_list_host.size());
    B->d_order = P.take<int>(count);
    B->static_bytes = P.off;
    // state region
    for (Member& M : B->mem) {
        const int m = M.m, n = M.n;
        M.x = P.take<double>(n);
        M.z = P.take<double>(n);
        M.ocone = P.take<double>((size_t)M.n_orth + M.n_soc);
        Outer& X = M.X;
        X.s = P.take<double>(n); X.p = P.take<double>(n); X.g = P.take<double>(n);
        X.q = P.take<double>(n); X.chat = P.take<double>(n); X.O = P.take<double>(n);
        X.w = P.take<double>(m); X.btil = P.take<double>(m);
        X.wp = P.take<double>(m); X.qp = P.take<double>(n);
        auto inner = [&](auto& V) {
            using T = std::remove_pointer_t<decltype(V.r)>;
            V.r = P.take<T>(m); V.u = P.take<T>(m); V.p = P.take<T>(m); V.sv = P.take<T>(m);
            V.au = P.take<T>(m); V.jinv = P.take<T>(m); V.t = P.take<T>(n); V.O2 = P.take<T>(n);
        };
        inner(M.V32);
        inner(M.V64);
    }
    B->d_p32 = P.take<IterParams<float>>(count);
    B->d_p64 = P.take<IterParams<double>>(count);
    B->d_ctl = P.take<Control>(count);
    B->d_head = P.take<int>(32);
    B->d_mailbox = P.take<int>(B->max_ctas);
    B->d_team_bar = P.take<unsigned long long>(B->max_ctas);
    B->d_team_part = P.take<double>((size_t)B->max_ctas * kMaxRed);
    B->d_team_err = P.take<int>(B->max_ctas);
    B->d_dense = P.take<double>(B->dense_m2 > 0 ? (size_t)B->max_ctas * 2 * B->dense_m2 : 1);
    B->total_bytes = P.off;
}

// Host preparation of every member (no device involved): validation,
// relabelling and images of each distinct A, b in relabelled order, norms,
// and the members in decreasing order of work.  On failure returns the code
// of the first failing member in member order and its index in *bad.
int prepare_members(Batch* B, int count, const acs_instance* members, int* bad) {
    // lanes per row are chosen for the smallest team (one 256-thread CTA,
    // 8 warps) so that any mapping can run
    const long long warps = 8;
    // members are independent: prepared on up to 16 host threads (a few
    // members stay on the caller), each taking the next unprepared member
    const int T = count >= 64 ? host::host_threads(1LL << 20) : 1;
    B->mem.resize(count);
    std::vector<int> rc(count, ACS_SOLVED);
    std::vector<Matrix> own(count);                      // built by the members that hold an A
    std::atomic<int> next{0};
    host::parallel_for(T, [&](int) {
        for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) {
            const acs_instance& I = members[i];
            if (I.share_A_with >= 0) {
                const int j = I.share_A_with;
                if (j >= i || I.m != members[j].m || I.n != members[j].n) { rc[i] = ACS_ERR_ARG; continue; }
                int root = j;                            // the member that holds the data
                while (members[root].share_A_with != -1) {
                    // a link that does not point back, an invalid one, or one to
                    // a member of other dimensions fails an earlier member, which
                    // is the one reported; the arrays along the chain are not
                    // read here (a member of other dimensions has arrays of
                    // other lengths)
                    const int up = members[root].share_A_with;
                    if (up < -1 || up >= root || members[up].m != I.m || members[up].n != I.n) {
                        rc[i] = ACS_ERR_ARG;
                        break;
                    }
                    root = up;
                }
                if (rc[i] != ACS_SOLVED) continue;
                rc[i] = host::validate(I.m, I.n, members[root].row_ptr, members[root].col, members[root].val,
                                       I.b, I.c, I.n_orthant, I.n_soc, I.soc_dims);
            } else {
                if (I.share_A_with < -1) { rc[i] = ACS_ERR_ARG; continue; }
                rc[i] = host::validate(I.m, I.n, I.row_ptr, I.col, I.val, I.b, I.c, I.n_orthant, I.n_soc,
                                       I.soc_dims);
                if (rc[i] != ACS_SOLVED) continue;
                if (host::build(I.m, I.n, I.row_ptr, I.col, I.val, I.b, I.c, I.n_orthant, I.n_soc, I.soc_dims,
                                warps, warps, own[i].H) != ACS_SOLVED) {
                    rc[i] = ACS_ERR_CSR;
                    continue;
                }
                own[i].stored = (long long)own[i].H.A.col.size();
            }
        }
    });
    // the first failing member, in member order
    for (int i = 0; i < count; ++i)
        if (rc[i] != ACS_SOLVED) {
            *bad = i;
            return rc[i];
        }
    // distinct matrices in member order
    std::vector<int> mat_of(count, -1);
    for (int i = 0; i < count; ++i) {
        if (members[i].share_A_with >= 0) {
            mat_of[i] = mat_of[members[i].share_A_with];
        } else {
            mat_of[i] = (int)B->mats.size();
            B->mats.push_back(std::move(own[i]));
        }
    }
    host::parallel_for(T, [&](int t) {
        const int i1 = (int)host::part_lo(count, t + 1, T);
        for (int i = (int)host::part_lo(count, t, T); i < i1; ++i) {
            const acs_instance& I = members[i];
            Member& M = B->mem[i];
            const Matrix& X = B->mats[mat_of[i]];
            M.m = I.m; M.n = I.n; M.n_orth = I.n_orthant; M.n_soc = I.n_soc; M.mat = mat_of[i];
            M.dense = host::dense_mode(B->set, I.m);
            M.nnz = X.stored;
            M.b.resize(I.m);
            for (int r = 0; r < I.m; ++r) M.b[r] = I.b[X.H.perm[r]];
            M.c.assign(I.c, I.c + I.n);
            M.soc_off.resize(I.n_soc + 1);
            M.soc_off[0] = I.n_orthant;
            for (int k = 0; k < I.n_soc; ++k) M.soc_off[k + 1] = M.soc_off[k] + I.soc_dims[k];
            double bn = 0, cn = 0;
            for (int r = 0; r < I.m; ++r) bn += I.b[r] * I.b[r];
            for (int j = 0; j < I.n; ++j) cn += I.c[j] * I.c[j];
            M.bnorm = sqrt(bn);
            M.cnorm = sqrt(cn);
        }
    });
    for (const Member& M : B->mem)
        if (M.dense) B->dense_m2 = std::max(B->dense_m2, (long long)M.m * M.m);
    // members in decreasing order of work (stored entries of A and A', plus vectors)
    B->order.resize(count);
    std::iota(B->order.begin(), B->order.end(), 0);
    std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b2) {
        const Member& x = B->mem[a];
        const Member& y = B->mem[b2];
        return 2 * x.nnz + 4LL * (x.m + x.n) > 2 * y.nnz + 4LL * (y.m + y.n);
    });
    return ACS_SOLVED;
}

// The host image of the static region (matrices, b, c, cone offsets, the
// conditioning list and the member order) at the offsets of layout().  The
// parts are disjoint: zeroed, then written, on up to 16 host threads.
void fill_image(Batch* B, host::raw_vector<char>& img) {
    const size_t bytes = B->static_bytes;
    img.resize(bytes);
    const int T = host::host_threads((long long)(bytes / 16));
    host::parallel_for(T, [&](int t) {
        const size_t a = (size_t)host::part_lo((long long)bytes, t, T);
        const size_t e = (size_t)host::part_lo((long long)bytes, t + 1, T);
        memset(img.data() + a, 0, e - a);
    });
    const size_t nm = B->mats.size(), nmem = B->mem.size();
    std::atomic<size_t> next{0};
    host::parallel_for(T, [&](int) {
        for (size_t k = next.fetch_add(1); k < nm + nmem; k = next.fetch_add(1)) {
            if (k < nm) {
                const Matrix& X = B->mats[k];
                image_sell(img, X.H.A, X.dA);
                image_sell(img, X.H.AT, X.dAT);
            } else {
                const Member& M = B->mem[k - nm];
                put_bytes(img.data(), M.db, M.b.data(), M.b.size());
                put_bytes(img.data(), M.dc, M.c.data(), M.c.size());
                put_bytes(img.data(), M.dsoc, M.soc_off.data(), M.soc_off.size());
            }
        }
    });
    put_bytes(img.data(), B->d_cond_list, B->cond_list_host.data(), B->cond_list_host.size());
    put_bytes(img.data(), B->d_order, B->order.data(), B->order.size());
}

void free_batch(Batch* B) {
    if (!B) return;
    drop_graph(B);
    if (B->pool) cudaFree(B->pool);
    B->pool = nullptr;
    for (auto& e : B->ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    B->stream = nullptr;
}

}  // namespace
}  // namespace acs

using acs::Batch;

extern "C" {

int acs_batch_create(int32_t count, const acs_instance* members, const acs_settings* settings,
                     const acs_batch_mapping* mapping, acs_batch** out, int32_t* bad_member) {
    using namespace acs;
    if (bad_member) *bad_member = -1;
    if (!out) return ACS_ERR_ARG;
    *out = nullptr;
    if (count <= 0 || !members) return ACS_ERR_ARG;
    acs_settings set;
    if (settings) set = *settings; else acs_settings_default(&set);
    if (!host::valid_settings(set)) return ACS_ERR_ARG;
    acs_batch_mapping map0 = mapping ? *mapping : acs_batch_mapping{1024, 1};
    if (!valid_mapping(map0)) return ACS_ERR_ARG;

    Batch* B = new (std::nothrow) Batch();
    if (!B) return ACS_ERR_OOM;
    B->count = count;
    B->set = set;
    B->device = set.device;
    if (set.n_cond_list > 0) B->cond_list_host.assign(set.cond_list, set.cond_list + set.n_cond_list);
    B->set.cond_list = nullptr;
    auto fail = [&](int rc, int i) {
        if (bad_member) *bad_member = i;
        free_batch(B);
        delete B;
        return rc;
    };

    {
        int bad = -1;
        const int rc = host::no_throw([&] { return prepare_members(B, count, members, &bad); });
        if (rc != ACS_SOLVED) return fail(rc, bad);
    }
    // the device is touched only once every member has passed the host checks
    if (cudaSetDevice(B->device) != cudaSuccess) return fail(ACS_ERR_CUDA, -1);
    if (cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, B->device) != cudaSuccess)
        return fail(ACS_ERR_CUDA, -1);
    {
        int bps = 0;                      // the most CTAs any mapping launches: 256-thread ones
        if (occupancy_for(256, &bps) != ACS_SOLVED) return fail(ACS_ERR_CUDA, -1);
        B->max_ctas = B->nsm * bps;
    }
    if (set.cuda_stream) {
        B->stream = (cudaStream_t)set.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(ACS_ERR_CUDA, -1);
        B->own_stream = true;
    }
    if (cudaEventCreate(&B->ev[0]) != cudaSuccess || cudaEventCreate(&B->ev[1]) != cudaSuccess)
        return fail(ACS_ERR_CUDA, -1);
    // device memory: one allocation, static region uploaded from a host image
    Pool dry;
    layout(B, dry);
    if (cudaMalloc(&B->pool, B->total_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ACS_ERR_OOM, -1);
    }
    {
        host::raw_vector<char> img;
        try {
            fill_image(B, img);
        } catch (...) {
            return fail(ACS_ERR_OOM, -1);
        }
        if (cudaMemcpy(B->pool, img.data(), B->static_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(ACS_ERR_CUDA, -1);
    }
    if (cudaMemsetAsync(B->pool + B->static_bytes, 0, B->total_bytes - B->static_bytes, B->stream) != cudaSuccess ||
        cudaStreamSynchronize(B->stream) != cudaSuccess)
        return fail(ACS_ERR_CUDA, -1);
    // turn the offsets into device addresses
    char* base = B->pool;
    for (Matrix& X : B->mats) {
        auto fin = [&](const host::HostSell& H, const DevSell& D, SellMat& S) {
            S.nrows = H.nrows; S.nslices = H.nslices; S.g = H.g;
            rebase_sell(D, base, S);
        };
        fin(X.H.A, X.dA, X.A);
        fin(X.H.AT, X.dAT, X.AT);
    }
    for (Member& M : B->mem) {
        M.db = rebase(M.db, base); M.dc = rebase(M.dc, base); M.dsoc = rebase(M.dsoc, base);
        M.x = rebase(M.x, base); M.z = rebase(M.z, base); M.ocone = rebase(M.ocone, base);
        Outer& X = M.X;
        X.s = rebase(X.s, base); X.p = rebase(X.p, base); X.g = rebase(X.g, base); X.q = rebase(X.q, base);
        X.chat = rebase(X.chat, base); X.O = rebase(X.O, base); X.w = rebase(X.w, base);
        X.btil = rebase(X.btil, base);
        X.wp = rebase(X.wp, base);
        X.qp = rebase(X.qp, base);
        auto inner = [&](auto& V) {
            V.r = rebase(V.r, base); V.u = rebase(V.u, base); V.p = rebase(V.p, base); V.sv = rebase(V.sv, base);
            V.au = rebase(V.au, base); V.jinv = rebase(V.jinv, base); V.t = rebase(V.t, base);
            V.O2 = rebase(V.O2, base);
        };
        inner(M.V32);
        inner(M.V64);
    }
    B->d_cond_list = rebase(B->d_cond_list, base);
    B->d_order = rebase(B->d_order, base);
    B->d_p32 = rebase(B->d_p32, base);
    B->d_p64 = rebase(B->d_p64, base);
    B->d_ctl = rebase(B->d_ctl, base);
    B->d_head = rebase(B->d_head, base);
    B->d_mailbox = rebase(B->d_mailbox, base);
    B->d_team_bar = rebase(B->d_team_bar, base);
    B->d_team_part = rebase(B->d_team_part, base);
    B->d_team_err = rebase(B->d_team_err, base);
    B->d_dense = rebase(B->d_dense, base);
    // the host images are no longer needed (keep the row relabelling)
    for (Matrix& X : B->mats) {
        std::vector<int> perm = std::move(X.H.perm);
        X.H = host::HostProblem();
        X.H.perm = std::move(perm);
    }
    for (Member& M : B->mem) {
        std::vector<double>().swap(M.b);
        std::vector<double>().swap(M.c);
        std::vector<int>().swap(M.soc_off);
    }
    const int rc = set_mapping(B, map0);
    if (rc != ACS_SOLVED) return fail(rc, -1);
    *out = reinterpret_cast<acs_batch*>(B);
    return ACS_SOLVED;
}

int acs_batch_set_mapping(acs_batch* h, const acs_batch_mapping* mapping) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !mapping) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    return acs::set_mapping(B, *mapping);
}

int acs_batch_solve_async(acs_batch* h, double tol, int32_t max_iter) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !(tol >= 0) || max_iter < 0) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    return acs::launch(B, tol, max_iter, true);
}

int acs_batch_results(acs_batch* h, int32_t* status, int32_t* iters, double* residuals) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
    int worst = ACS_SOLVED;
    for (int i = 0; i < B->count; ++i) {
        const acs::Control& C = B->ctl_host[i];
        const int s = acs::member_status(C);
        if (status) status[i] = s;
        if (iters) iters[i] = C.l;
        if (residuals) {
            for (int k = 0; k < 6; ++k) residuals[8 * i + k] = C.res[k];
            residuals[8 * i + 6] = (double)C.cg_iters;
            residuals[8 * i + 7] = (double)C.switched_at;
        }
        if (s < 0 && worst >= 0) worst = s;
        else if (s == ACS_MAX_ITER && worst == ACS_SOLVED) worst = ACS_MAX_ITER;
    }
    return worst;
}

int acs_batch_solve(acs_batch* h, double tol, int32_t max_iter) {
    const int rc = acs_batch_solve_async(h, tol, max_iter);
    if (rc != ACS_SOLVED) return rc;
    return acs_batch_results(h, nullptr, nullptr, nullptr);
}

int acs_batch_get(acs_batch* h, int32_t i, double* x, double* y, double* s, int32_t* iters, double* residuals) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || i < 0 || i >= B->count) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    const acs::Member& M = B->mem[i];
    acs::Control C;
    cudaStream_t st = B->stream;
    std::vector<double> w;
    if (cudaMemcpyAsync(&C, B->d_ctl + i, sizeof(C), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ACS_ERR_CUDA;
    if (x && cudaMemcpyAsync(x, M.x, sizeof(double) * M.n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (s && cudaMemcpyAsync(s, M.z, sizeof(double) * M.n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return ACS_ERR_CUDA;
    if (y) {
        w.resize(M.m);
        if (cudaMemcpyAsync(w.data(), M.X.w, sizeof(double) * M.m, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return ACS_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return ACS_ERR_CUDA;
    if (y) {
        const std::vector<int>& perm = B->mats[M.mat].H.perm;
        for (int r = 0; r < M.m; ++r) y[perm[r]] = w[r] / B->set.mu;
    }
    if (iters) *iters = C.l;
    if (residuals) {
        for (int k = 0; k < 6; ++k) residuals[k] = C.res[k];
        residuals[6] = (double)C.cg_iters;
        residuals[7] = (double)C.switched_at;
    }
    return acs::member_status(C);
}

int acs_batch_autotune(acs_batch* h, int32_t max_iter, acs_batch_mapping* chosen, double* ms) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || max_iter <= 0) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    const acs_batch_mapping keep = B->map;
    double best = INFINITY;
    acs_batch_mapping best_map = keep;
    int idx = 0;
    for (int th : acs::kThreadChoices)
        for (int g : acs::kTeamChoices) {
            const acs_batch_mapping cand{th, g};
            double t = -1.0;
            if (acs::set_mapping(B, cand) == ACS_SOLVED) {
                // one untimed run (warms caches and the launch), then a timed one
                int rc = acs::launch(B, 0.0, max_iter, false);
                if (rc == ACS_SOLVED) rc = acs::launch(B, 0.0, max_iter, false);
                float f = 0.f;
                if (rc == ACS_SOLVED && cudaEventSynchronize(B->ev[1]) == cudaSuccess &&
                    cudaEventElapsedTime(&f, B->ev[0], B->ev[1]) == cudaSuccess) {
                    t = f;
                    if (t < best) { best = t; best_map = cand; }
                }
            }
            if (ms) ms[idx] = t;
            ++idx;
        }
    if (!(best < INFINITY)) {
        acs::set_mapping(B, keep);
        return ACS_ERR_CUDA;
    }
    const int rc = acs::set_mapping(B, best_map);
    if (chosen) *chosen = best_map;
    return rc;
}

int acs_batch_last_ms(acs_batch* h, double* ms) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !ms) return ACS_ERR_ARG;
    float f = 0.f;
    if (cudaEventSynchronize(B->ev[1]) != cudaSuccess || cudaEventElapsedTime(&f, B->ev[0], B->ev[1]) != cudaSuccess)
        return ACS_ERR_CUDA;
    *ms = (double)f;
    return ACS_SOLVED;
}

int acs_batch_info(acs_batch* h, long long* out8, long long* counters6) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !out8) return ACS_ERR_ARG;
    long long sm = 0, sn = 0, nnz = 0;
    for (const auto& M : B->mem) { sm += M.m; sn += M.n; }
    for (const auto& X : B->mats) nnz += X.stored;
    out8[0] = B->count;
    out8[1] = (long long)B->mats.size();
    out8[2] = sm;
    out8[3] = sn;
    out8[4] = nnz;
    out8[5] = B->grid / B->map.team_ctas;
    out8[6] = B->grid;
    out8[7] = B->last_graph ? 1 : 0;
    if (counters6) {
        if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
        for (int k = 0; k < 6; ++k) counters6[k] = 0;
        for (const auto& C : B->ctl_host) {
            counters6[0] += C.n_cg_A; counters6[1] += C.n_cg_AT; counters6[2] += C.n_64_A;
            counters6[3] += C.n_64_AT; counters6[4] += C.n_cond; counters6[5] += C.n_checks;
        }
    }
    return ACS_SOLVED;
}

int acs_batch_counters(acs_batch* h, long long* out) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !out) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
    for (int i = 0; i < B->count; ++i) {
        const acs::Control& C = B->ctl_host[i];
        long long* o = out + 8 * (size_t)i;
        o[0] = C.n_cg_A; o[1] = C.n_cg_AT; o[2] = C.n_64_A; o[3] = C.n_64_AT;
        o[4] = C.n_cond; o[5] = C.n_checks; o[6] = C.n_dense_solve; o[7] = C.n_dense_factor;
    }
    return ACS_SOLVED;
}

int acs_batch_member_ms(acs_batch* h, double* ms) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !ms) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
    for (int i = 0; i < B->count; ++i) {
        unsigned long long t = 0;
        for (int k = 0; k < acs::PH_COUNT; ++k) t += B->ctl_host[i].phase_ns[k];
        ms[i] = (double)t * 1e-6;
    }
    return ACS_SOLVED;
}

int acs_batch_phase_ms(acs_batch* h, int32_t i, double* ms, long long* count, int32_t n) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B || !ms || !count || n < acs::PH_COUNT || i < -1 || i >= B->count) return ACS_ERR_ARG;
    if (cudaSetDevice(B->device) != cudaSuccess) return ACS_ERR_CUDA;
    if (acs::fetch_controls(B) != ACS_SOLVED) return ACS_ERR_CUDA;
    for (int k = 0; k < acs::PH_COUNT; ++k) {
        ms[k] = 0.0;
        count[k] = 0;
    }
    for (int j = (i < 0 ? 0 : i); j < (i < 0 ? B->count : i + 1); ++j)
        for (int k = 0; k < acs::PH_COUNT; ++k) {
            ms[k] += (double)B->ctl_host[j].phase_ns[k] * 1e-6;
            count[k] += (long long)B->ctl_host[j].phase_n[k];
        }
    return acs::PH_COUNT;
}

int acs_debug_batch_image(int32_t count, const acs_instance* members, const acs_settings* settings,
                          uint64_t* hash, int64_t* static_bytes, int32_t* bad_member) {
    using namespace acs;
    if (bad_member) *bad_member = -1;
    if (count <= 0 || !members || !hash || !static_bytes) return ACS_ERR_ARG;
    Batch B;
    if (settings) B.set = *settings; else acs_settings_default(&B.set);
    if (!host::valid_settings(B.set)) return ACS_ERR_ARG;
    if (B.set.n_cond_list > 0) B.cond_list_host.assign(B.set.cond_list, B.set.cond_list + B.set.n_cond_list);
    B.set.cond_list = nullptr;
    B.count = count;
    int bad = -1;
    const int rc = host::no_throw([&] { return prepare_members(&B, count, members, &bad); });
    if (rc != ACS_SOLVED) {
        if (bad_member) *bad_member = bad;
        return rc;
    }
    B.max_ctas = 152 * 8;           // sizes only the state region, which the image does not hold
    Pool dry;
    layout(&B, dry);
    host::raw_vector<char> img;
    if (host::no_throw([&] { fill_image(&B, img); return ACS_SOLVED; }) != ACS_SOLVED) return ACS_ERR_OOM;
    uint64_t h = 1469598103934665603ull;          // FNV-1a
    for (char ch : img) {
        h ^= (unsigned char)ch;
        h *= 1099511628211ull;
    }
    *hash = h;
    *static_bytes = (int64_t)B.static_bytes;
    return ACS_SOLVED;
}

void acs_batch_destroy(acs_batch* h) {
    Batch* B = reinterpret_cast<Batch*>(h);
    if (!B) return;
    cudaSetDevice(B->device);
    if (B->stream) cudaStreamSynchronize(B->stream);
    acs::free_batch(B);
    delete B;
}

}  // extern "C"
