// serve.cu -- continuous-batching solve server (serve_create / submit / poll).
//
// A server thread owns a side stream and two lane streams.  On each lane's
// stream it advances that lane's resident requests ("slots": a slot's matrix,
// right-hand sides and Krylov state stay on the device) by a chunk of CG
// iterations in shared launches -- the batched kernels of batched.cuh over a
// table of the lane's iterating slots; medium requests (n k2 <= 2^20) have a
// lane of their own, so they do not iterate at the pace of the largest ones.  While a chunk
// runs, pending requests are admitted on the side stream as slots and memory
// allow: device assembly, SELL conversion, Dirichlet lift and the start of
// their recurrences, allocated from a stream-ordered pool and charged against
// the memory budget.  A chunk ends after iters_per_step iterations (adaptive by
// default: about 10 ms of the resident set's iterations) or as soon
// as a slot's columns have all stopped; the thread then services those slots
// (fp32 recurrences: the reliable update -- x += d and r = b - A x in fp64,
// the fp64 test, residual replacement; fp64 recurrences: the true-residual
// check), retires finished ones (x copied to the caller's host buffer, memory
// freed), and rebuilds the table with the new arrivals.  A slot's arithmetic
// depends only on its own data, so its result is the same alone and in a mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "batched.cuh"

namespace gb {

constexpr double CHUNK_MS = 10.0;  // target length of a chunk in adaptive mode

static bool log_on() {
    static int v = -1;
    if (v < 0) { const char *e = getenv("GBPCG_LOG"); v = (e && *e && *e != '0') ? 1 : 0; }
    return v == 1;
}

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SReq {
    uint64_t ticket;
    ServeRequest r;
    std::vector<double> coef;
    double t_submit;
};

// SL_PWAIT: admitted, waiting for the next persistent launch; SL_PRUN: in one
enum { SL_ITER = 0, SL_SERVICE = 1, SL_DONE = 2, SL_PWAIT = 3, SL_PRUN = 4 };

struct Slot {
    SReq q;
    gb_fem_system *sys = nullptr;
    gb_sell *A = nullptr;
    int64_t n = 0;
    int k = 1, kw = 1;
    bool ru = true;
    int ptier = 0;  // persistent tier solving it (1 one block, 2 one cluster), 0 = the lock-step loop
    int lane = 0;   // lock-step lane: 1 for n k2 <= 2^GB_SERVE_MEDIUM_LOG2, else 0
    double *B64 = nullptr, *X64 = nullptr, *R64 = nullptr;
    void *X = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr;
    double *cd = nullptr;
    long long *ci = nullptr;
    int *cs = nullptr;
    ColState c{};
    std::vector<void *> bufs;  // engine-owned device buffers of this slot
    std::vector<int> fin;      // per column: 1 = final
    std::vector<int> fstat;    // final status per column
    std::vector<double> rel, best;
    std::vector<int> stalls;
    int updates = 0;
    int state = SL_ITER;
    int active = 0;            // columns iterating
    double t_admit = 0.0;
    size_t bytes = 0;
    int units = 1;
    int64_t rows_per_unit = 1;
};

}  // namespace gb

struct gb_server {
    ServeOptions opt{};
    int dev = 0;
    // One lock-step loop per lane, on a stream of its own with its own system
    // table: lane 0 takes the requests above 2^GB_SERVE_MEDIUM_LOG2 elements
    // (n k2) and the service steps, lane 1 the medium ones, so that a medium
    // request's iterations do not wait for the largest requests' iterations.
    struct Lane {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // timing of a chunk (adaptive chunk length)
        gb::BSys *d_sys = nullptr;
        int *d_unit_sys = nullptr;
        gb::BGlobal *d_G = nullptr;
        double *d_partials = nullptr;
        size_t cap_umap = 0, cap_part = 0;
        int ips = 16;  // iterations of the next chunk (adaptive mode)
    };
    static constexpr int NLANES = 2;
    Lane ln[NLANES];
    cudaStream_t side_st = nullptr;
    struct PLaunch {  // one persistent launch, on a stream of its own
        std::vector<gb::Slot *> slots;
        gb::BSys *d_tab = nullptr;
        int *d_list = nullptr;
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
    };
    std::vector<std::unique_ptr<PLaunch>> plaunch;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<gb::SReq> inbox;
    std::map<uint64_t, ServeResult> results;
    uint64_t next_ticket = 1;
    bool stopping = false;
    // accounting (server thread; read under mu for stats)
    ServeStats stats{};
    size_t in_use = 0, peak = 0;
    size_t slot_bytes_acc = 0;  // bytes allocated while admitting the current slot
    std::unordered_map<void *, size_t> sizes;
    gb_allocator alloc{};  // what the slots' assembly and SELL build allocate through (srv_alloc)
    gb_allocator user{};   // the caller's allocator (serve_create), or none: the stream-ordered pool
    int *d_mask = nullptr;  // column masks of the service step (lane 0's stream)
    // single-slot buffers used while admitting (side stream)
    gb::BSys *d_sys1 = nullptr;
    int *d_unit1 = nullptr, *d_mask1 = nullptr;
    double *d_partials1 = nullptr;
    size_t cap_umap1 = 0, cap_part1 = 0;
    std::vector<std::unique_ptr<gb::Slot>> slots;
    std::deque<gb::SReq> pending;
    int fatal = GB_OK;
    std::string fatal_msg;
};

using namespace gb;

// ------------------------------------------------------------- allocator --
// Allocations on the side stream, counted per slot: through the caller's
// allocator when serve_create was given one, else from the stream-ordered pool.
static void *srv_alloc(void *ctx, size_t bytes, void *stream) {
    gb_server *s = (gb_server *)ctx;
    void *p = nullptr;
    if (s->user.alloc) {
        p = s->user.alloc(s->user.ctx, bytes, stream);
        if (!p) return nullptr;
    } else if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) {
        return nullptr;
    }
    s->sizes[p] = bytes;
    s->in_use += bytes;
    s->slot_bytes_acc += bytes;
    s->peak = std::max(s->peak, s->in_use);
    return p;
}
static void srv_free(void *ctx, void *p, void *stream) {
    gb_server *s = (gb_server *)ctx;
    if (!p) return;
    auto it = s->sizes.find(p);
    if (it != s->sizes.end()) {
        s->in_use -= it->second;
        s->sizes.erase(it);
    }
    if (s->user.free) s->user.free(s->user.ctx, p, stream);
    else cudaFreeAsync(p, (cudaStream_t)stream);
}

template <class T>
static int srv_take(gb_server *s, Slot &sl, T **p, size_t n) {
    void *q = srv_alloc(s, std::max<size_t>(n * sizeof(T), 256), s->side_st);
    if (!q) { set_error("serve: device allocation of %zu bytes failed", n * sizeof(T)); return GB_ENOMEM; }
    sl.bufs.push_back(q);
    *p = (T *)q;
    return GB_OK;
}

static BSys desc_of(const Slot &sl, int unit0) {
    BSys S{};
    S.A = sl.A->view();
    S.val = sl.ru ? (const void *)sl.A->val32 : (const void *)sl.A->val;
    S.X = sl.X; S.R = sl.R; S.P = sl.P; S.Q = sl.Q;
    S.B64 = sl.B64; S.X64 = sl.X64; S.R64 = sl.R64;
    S.c = sl.c;
    S.k = sl.k; S.kw = sl.kw;
    S.unit0 = unit0;
    S.nunits = sl.units;
    S.rows_per_unit = sl.rows_per_unit;
    S.ticket = 0;
    S.active = sl.active;
    return S;
}

// device bytes one request will hold (upper estimate from its spec)
static size_t estimate_bytes(const ServeRequest &r, bool ru) {
    const int64_t S = (int64_t)r.spec.degree * r.spec.cells + 1;
    int64_t nd = 1, nf = 1;
    for (int d = 0; d < r.spec.dim; ++d) { nd *= S; nf *= (S - 2); }
    const double per_row = r.spec.dim == 2 ? (r.spec.degree == 1 ? 9.0 : 25.0) : (r.spec.degree == 1 ? 15.0 : 65.0);
    const double nnz = per_row * nf;
    const double nb = (double)(nd - nf);
    double b = nnz * 12.0 * 1.05           // CSR
               + nnz * 1.45 * (4 + 8 + (ru ? 4 : 0))  // SELL (padding bound)
               + nf * 60.0                  // row pointers, maps, diag, dinv, perm
               + nb * 16.0 + 4.0 * per_row * nb   // K_IB, boundary maps
               + (double)nf * r.k * (ru ? (3 * 8 + 4 * 4) : 5 * 8)  // vectors
               + (double)nb * r.k * 8 + (double)nf * r.k * 8     // lift temporaries
               + 65536;
    return (size_t)b;
}

static void finish(gb_server *s, const SReq &q, int status, const Slot *sl) {
    ServeResult R{};
    R.status = status;
    R.k = q.r.k;
    if (sl) {
        R.n = sl->n;
        R.updates = sl->updates;
        R.bytes = (double)sl->bytes;
        R.queue_ms = sl->t_admit - q.t_submit;
    }
    R.latency_ms = now_ms() - q.t_submit;
    std::lock_guard<std::mutex> lk(s->mu);
    s->results[q.ticket] = R;
    if (status == GB_TOO_LARGE && !sl) s->stats.rejected += 1;
    s->stats.completed += 1;
}

static void release_slot(gb_server *s, Slot &sl) {
    for (void *p : sl.bufs) srv_free(s, p, s->side_st);
    sl.bufs.clear();
    if (sl.A) { sell_destroy(sl.A); sl.A = nullptr; }
    if (sl.sys) { fem_system_destroy(sl.sys); sl.sys = nullptr; }
}

// grow a device buffer owned by the engine (not charged to any slot)
template <class T>
static int grow(gb_server *s, T **p, size_t *cap, size_t need, cudaStream_t st) {
    if (*p && *cap >= need) return GB_OK;
    if (*p) { cudaStreamSynchronize(st); cudaFree(*p); *p = nullptr; }
    size_t c = std::max<size_t>(need, 1024);
    GB_CHECK_CUDA(cudaMalloc((void **)p, c * sizeof(T)));
    *cap = c;
    return GB_OK;
}

// Requests up to n * k2 <= 2^15 (k2: the power of two >= k) are solved by one
// block each of k_bpersist, and, with ServeOptions.cluster_lane, requests up
// to n * k2 <= 2^16 by one 8-block cluster each of k_bcluster: such a request
// works through its iterations at the pace of its own SMs instead of in
// lock-step with the largest resident requests (which pays for the smallest
// ones; a cluster's 8 SMs make a medium request slower than the lock-step
// loop over all SMs unless many of them are resident).  Returns the tier
// (0: lock-step loop).
#ifndef GB_SERVE_PERSIST_LOG2
#define GB_SERVE_PERSIST_LOG2 15
#endif
static int serve_persist_tier(int64_t n, int k, bool ru, bool cluster_lane) {
    int kp = 1;
    while (kp < k) kp <<= 1;
    if (n * kp <= (ru ? ((int64_t)1 << GB_SERVE_PERSIST_LOG2) : PERSIST_MAX_ELEMS)) return 1;
    if (cluster_lane && n * kp <= CLUSTER_MAX_ELEMS) return 2;
    return 0;
}

// Lock-step lane of a request: medium requests (n k2 <= 2^GB_SERVE_MEDIUM_LOG2)
// iterate in lane 1, larger ones in lane 0, each lane in launches of its own
// on its own stream, so a medium request advances at the pace of the medium
// requests' iterations rather than the largest requests' (160 seeded
// requests of 2D/3D P1/P2 meshes with 1-8 right-hand sides: medium requests
// waited 16 x their one-at-a-time time at the median with a single lane,
// 7.5 x with two).
#ifndef GB_SERVE_MEDIUM_LOG2
#define GB_SERVE_MEDIUM_LOG2 20
#endif
static int serve_lane(int64_t n, int k) {
    int kp = 1;
    while (kp < k) kp <<= 1;
    return n * kp <= ((int64_t)1 << GB_SERVE_MEDIUM_LOG2) ? 1 : 0;
}

// --------------------------------------------------------------- admit --
static int admit(gb_server *s, SReq &q, std::unique_ptr<Slot> &out) {
    const bool ru = s->opt.precision != GB_F64;
    auto sl = std::make_unique<Slot>();
    Slot &L = *sl;
    L.q = q;
    L.ru = ru;
    L.k = q.r.k;
    L.kw = 1;
    while (L.kw < L.k) L.kw <<= 1;
    s->slot_bytes_acc = 0;
    cudaStream_t st = s->side_st;
    int rc = fem_assemble(&q.r.spec, &s->alloc, st, &L.sys);
    if (rc == GB_OK) rc = csr_to_sell(L.sys, 32, 256, ru ? (GB_VAL_F64 | GB_VAL_F32) : GB_VAL_F64, &s->alloc, st, &L.A);
    if (rc != GB_OK) { L.bytes = s->slot_bytes_acc; release_slot(s, L); return rc; }
    gb_fem_info fi{};
    fem_system_info(L.sys, &fi);
    L.n = fi.n_free;
    const size_t nk = (size_t)L.n * L.k;
    double *gB = nullptr, *bfull = nullptr;
    rc = srv_take(s, L, &L.B64, nk);
    if (rc == GB_OK) rc = srv_take(s, L, &L.X64, nk);
    if (rc == GB_OK) rc = srv_take(s, L, &L.R64, nk);
    if (rc == GB_OK) rc = srv_take(s, L, &gB, (size_t)fi.n_bnd * L.k);
    if (rc == GB_OK) rc = srv_take(s, L, &bfull, nk);
    if (rc == GB_OK) {
        if (ru) {
            float *X, *R, *P, *Q;
            rc = srv_take(s, L, &X, nk);
            if (rc == GB_OK) rc = srv_take(s, L, &R, nk);
            if (rc == GB_OK) rc = srv_take(s, L, &P, nk);
            if (rc == GB_OK) rc = srv_take(s, L, &Q, nk);
            L.X = X; L.R = R; L.P = P; L.Q = Q;
        } else {
            double *P, *Q;
            rc = srv_take(s, L, &P, nk);
            if (rc == GB_OK) rc = srv_take(s, L, &Q, nk);
            L.X = L.X64; L.R = L.R64; L.P = P; L.Q = Q;
        }
    }
    if (rc == GB_OK) rc = srv_take(s, L, &L.cd, (size_t)10 * KMAX);
    if (rc == GB_OK) rc = srv_take(s, L, &L.ci, (size_t)KMAX);
    if (rc == GB_OK) rc = srv_take(s, L, &L.cs, (size_t)2 * KMAX);
    if (rc != GB_OK) { L.bytes = s->slot_bytes_acc; release_slot(s, L); return rc; }
    L.c.rho = L.cd; L.c.pq = L.cd + KMAX; L.c.alpha = L.cd + 2 * KMAX; L.c.beta = L.cd + 3 * KMAX;
    L.c.rr = L.cd + 4 * KMAX; L.c.bb = L.cd + 5 * KMAX; L.c.thresh = L.cd + 6 * KMAX; L.c.scale = L.cd + 7 * KMAX;
    L.c.pz = L.cd + 8 * KMAX; L.c.target = L.cd + 9 * KMAX;
    L.c.it = L.ci;
    L.c.done = L.cs; L.c.status = L.cs + KMAX;
    auto fail = [&](const char *what, cudaError_t e) {
        set_error("serve admit: %s: %s", what, cudaGetErrorString(e));
        L.bytes = s->slot_bytes_acc;
        release_slot(s, L);
        return GB_ECUDA;
    };
    cudaError_t e = cudaMemsetAsync(L.cd, 0, sizeof(double) * 10 * KMAX, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.ci, 0, sizeof(long long) * KMAX, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.cs, 0, sizeof(int) * 2 * KMAX, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.X64, 0, sizeof(double) * nk, st);
    if (e != cudaSuccess) return fail("memset", e);
    // right-hand sides: b = -K_IB g_B in free-dof order, then permuted
    if (q.r.h_gB) {
        e = cudaMemcpyAsync(gB, q.r.h_gB, sizeof(double) * fi.n_bnd * L.k, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail("gB copy", e);
    } else {
        rc = fem_dirichlet(L.sys, q.r.gid, q.coef.empty() ? nullptr : q.coef.data(), L.k, 0, gB, st);
        if (rc != GB_OK) { L.bytes = s->slot_bytes_acc; release_slot(s, L); return rc; }
    }
    rc = fem_lift_rhs(L.sys, gB, L.k, bfull, st);
    if (rc != GB_OK) { L.bytes = s->slot_bytes_acc; release_slot(s, L); return rc; }
    ::gb::count_launches(1);
    k_gather_rows<<<stride_grid((int64_t)nk, 256, 8), 256, 0, st>>>(L.n, L.k, L.A->perm, bfull, L.B64);
    // single-slot table: initial residual (x0 = 0), norms, thresholds
    L.units = units_of_rows(L.n, &L.rows_per_unit);
    GB_TRY(grow(s, &s->d_partials1, &s->cap_part1, (size_t)L.units * 3 * KMAX, st));
    std::vector<int> umap(L.units, 0);
    GB_TRY(grow(s, &s->d_unit1, &s->cap_umap1, (size_t)L.units, st));
    L.active = 0;
    BSys d1 = desc_of(L, 0);
    e = cudaMemcpyAsync(s->d_sys1, &d1, sizeof(BSys), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_unit1, umap.data(), sizeof(int) * L.units, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail("table", e);
    ::gb::count_launches(1);
    k_bresid<<<L.units, NT, 0, st>>>(s->d_sys1, s->d_unit1, s->d_partials1, 1, 1, s->opt.tol);
    std::vector<double> bb(L.k), rr(L.k);
    e = cudaMemcpyAsync(bb.data(), L.c.bb, sizeof(double) * L.k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail("init residual", e);
    srv_free(s, gB, st);
    srv_free(s, bfull, st);
    L.bufs.erase(std::remove(L.bufs.begin(), L.bufs.end(), (void *)gB), L.bufs.end());
    L.bufs.erase(std::remove(L.bufs.begin(), L.bufs.end(), (void *)bfull), L.bufs.end());
    L.fin.assign(L.k, 0);
    L.fstat.assign(L.k, GB_OK);
    L.rel.assign(L.k, 1.0);
    L.best.assign(L.k, 1.0);
    L.stalls.assign(L.k, 0);
    std::vector<int> mask(KMAX, 0);
    std::vector<double> target(KMAX, 0.0);
    for (int j = 0; j < L.k; ++j) {
        if (bb[j] == 0.0) { L.fin[j] = 1; L.rel[j] = 0.0; continue; }  // zero data: x = 0
        mask[j] = ru ? 2 : 1;
        target[j] = 0.25 * s->opt.tol * s->opt.tol * bb[j];
    }
    L.ptier = serve_persist_tier(L.n, L.k, ru, s->opt.cluster_lane != 0);
    L.lane = serve_lane(L.n, L.k);
    if (L.ptier) {
        // small or medium request: solved whole by one block (or one cluster)
        // of the next persistent launch (launch_persistent), not in the
        // lock-step loop
        L.active = 0;
        L.state = SL_PWAIT;
        L.bytes = s->slot_bytes_acc;
        L.t_admit = now_ms();
        out = std::move(sl);
        return GB_OK;
    }
    e = cudaMemcpyAsync(s->d_mask1, mask.data(), sizeof(int) * KMAX, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.c.target, target.data(), sizeof(double) * KMAX, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail("mask", e);
    if (ru) {
        ::gb::count_launches(2);
        k_breplace<<<L.units, NT, 0, st>>>(s->d_sys1, s->d_unit1, s->d_partials1, s->d_mask1, 0.01);
        k_breplace_p<<<L.units, NT, 0, st>>>(s->d_sys1, s->d_unit1, s->d_mask1);
    } else {
        ::gb::count_launches(1);
        k_bstart<double><<<L.units, NT, 0, st>>>(s->d_sys1, s->d_unit1, s->d_partials1, s->d_mask1);
    }
    std::vector<int> done(L.k);
    e = cudaMemcpyAsync(done.data(), L.c.done, sizeof(int) * L.k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail("start", e);
    for (int j = 0; j < L.k; ++j) L.active += (!L.fin[j] && !done[j]) ? 1 : 0;
    L.state = L.active ? SL_ITER : SL_SERVICE;
    L.bytes = s->slot_bytes_acc;
    L.t_admit = now_ms();
    out = std::move(sl);
    return GB_OK;
}

// --------------------------------------------------------- retire / service --
static void retire(gb_server *s, Slot &L, int status) {
    // x back in free-dof order into the caller's buffer
    double *xo = nullptr;
    int rc = srv_take(s, L, &xo, (size_t)L.n * L.k);
    cudaError_t e = cudaSuccess;
    if (rc == GB_OK) {
        ::gb::count_launches(1);
        k_scatter_rows<<<stride_grid(L.n * L.k, 256, 8), 256, 0, s->side_st>>>(L.n, L.k, L.A->perm, L.X64, xo);
        e = cudaMemcpyAsync(L.q.r.h_x, xo, sizeof(double) * L.n * L.k, cudaMemcpyDeviceToHost, s->side_st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->side_st);
    }
    if (rc != GB_OK || e != cudaSuccess) status = rc != GB_OK ? rc : GB_ECUDA;
    std::vector<long long> it(L.k, 0);
    cudaMemcpy(it.data(), L.c.it, sizeof(long long) * L.k, cudaMemcpyDeviceToHost);
    release_slot(s, L);
    ServeResult R{};
    R.status = status;
    R.k = L.k;
    R.n = L.n;
    for (int j = 0; j < L.k; ++j) {
        R.iterations = std::max<int64_t>(R.iterations, it[j]);
        R.relres = std::max(R.relres, L.rel[j]);
    }
    R.updates = L.updates;
    R.bytes = (double)L.bytes;
    R.queue_ms = L.t_admit - L.q.t_submit;
    R.latency_ms = now_ms() - L.q.t_submit;
    std::lock_guard<std::mutex> lk(s->mu);
    s->results[L.q.ticket] = R;
    s->stats.completed += 1;
    s->stats.resident -= 1;
    L.state = SL_DONE;
}

// Slots whose columns have all stopped: fp64 correction and residual, the
// fp64 test per column, then either final or re-armed (replacement / restart).
static int service(gb_server *s, std::vector<Slot *> &sv) {
    if (sv.empty()) return GB_OK;
    cudaStream_t st = s->ln[0].st;
    const bool ru = s->opt.precision != GB_F64;
    std::vector<BSys> tab;
    std::vector<int> umap;
    for (size_t i = 0; i < sv.size(); ++i) {
        tab.push_back(desc_of(*sv[i], (int)umap.size()));
        for (int u = 0; u < sv[i]->units; ++u) umap.push_back((int)i);
    }
    GB_TRY(grow(s, &s->ln[0].d_partials, &s->ln[0].cap_part, umap.size() * 3 * KMAX, st));
    GB_TRY(grow(s, &s->ln[0].d_unit_sys, &s->ln[0].cap_umap, umap.size(), st));
    std::vector<int> mask(tab.size() * KMAX, 0);
    for (size_t i = 0; i < sv.size(); ++i)
        for (int j = 0; j < sv[i]->k; ++j) mask[i * KMAX + j] = sv[i]->fin[j] ? 0 : 1;
    GB_CHECK_CUDA(cudaMemcpyAsync(s->ln[0].d_sys, tab.data(), sizeof(BSys) * tab.size(), cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemcpyAsync(s->ln[0].d_unit_sys, umap.data(), sizeof(int) * umap.size(), cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemcpyAsync(s->d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
    const int U = (int)umap.size();
    if (ru) {
        // scale = 1: X64 += D for the columns that were iterating
        for (auto *L : sv) {
            std::vector<double> one(KMAX, 1.0);
            GB_CHECK_CUDA(cudaMemcpyAsync(L->c.scale, one.data(), sizeof(double) * KMAX, cudaMemcpyHostToDevice, st));
        }
        ::gb::count_launches(1);
        k_bcorrect<<<U, NT, 0, st>>>(s->ln[0].d_sys, s->ln[0].d_unit_sys, s->d_mask);
    }
    ::gb::count_launches(1);
    k_bresid<<<U, NT, 0, st>>>(s->ln[0].d_sys, s->ln[0].d_unit_sys, s->ln[0].d_partials, 0, 0, s->opt.tol);
    GB_CHECK_CUDA(cudaGetLastError());
    // decide per column
    bool any = false;
    for (size_t i = 0; i < sv.size(); ++i) {
        Slot &L = *sv[i];
        std::vector<double> rr(L.k), bb(L.k);
        std::vector<int> stat(L.k);
        std::vector<long long> it(L.k);
        GB_CHECK_CUDA(cudaMemcpyAsync(rr.data(), L.c.rr, sizeof(double) * L.k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(bb.data(), L.c.bb, sizeof(double) * L.k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(stat.data(), L.c.status, sizeof(int) * L.k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(it.data(), L.c.it, sizeof(long long) * L.k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        L.updates += ru ? 1 : 0;
        for (int j = 0; j < L.k; ++j) {
            const int m = mask[i * KMAX + j];
            if (!m) continue;
            const double rel = bb[j] > 0 ? std::sqrt(rr[j] / bb[j]) : 0.0;
            L.rel[j] = rel;
            int nm = 0;
            if (rel <= s->opt.tol) { L.fin[j] = 1; L.fstat[j] = GB_OK; }
            else if (stat[j] == ST_MAXIT || it[j] >= s->opt.max_iter) { L.fin[j] = 1; L.fstat[j] = GB_NOT_CONVERGED; }
            else {
                if (rel < 0.9 * L.best[j]) { L.best[j] = rel; L.stalls[j] = 0; }
                else if (++L.stalls[j] >= 4) { L.fin[j] = 1; L.fstat[j] = GB_NOT_CONVERGED; }
                if (!L.fin[j]) nm = (stat[j] == ST_BREAK) ? 2 : 1;  // breakdown: fresh direction
            }
            mask[i * KMAX + j] = nm;
            any |= nm != 0;
            if (log_on())
                fprintf(stderr, "[gbpcg serve] ticket %llu col %d: it %lld status %d rel %.3e best %.3e stalls %d -> %s\n",
                        (unsigned long long)L.q.ticket, j, it[j], stat[j], rel, L.best[j], L.stalls[j],
                        L.fin[j] ? (L.fstat[j] == GB_OK ? "converged" : "stopped") : (nm == 2 ? "fresh start" : "replace"));
        }
    }
    if (any) {
        GB_CHECK_CUDA(cudaMemcpyAsync(s->d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
        if (ru) {
            ::gb::count_launches(2);
            k_breplace<<<U, NT, 0, st>>>(s->ln[0].d_sys, s->ln[0].d_unit_sys, s->ln[0].d_partials, s->d_mask, 0.01);
            k_breplace_p<<<U, NT, 0, st>>>(s->ln[0].d_sys, s->ln[0].d_unit_sys, s->d_mask);
        } else {
            // fp64 recurrence: restart from the true residual (R64 already holds it)
            ::gb::count_launches(1);
            k_bstart<double><<<U, NT, 0, st>>>(s->ln[0].d_sys, s->ln[0].d_unit_sys, s->ln[0].d_partials, s->d_mask);
        }
        GB_CHECK_CUDA(cudaGetLastError());
    }
    for (size_t i = 0; i < sv.size(); ++i) {
        Slot &L = *sv[i];
        std::vector<int> done(L.k);
        GB_CHECK_CUDA(cudaMemcpyAsync(done.data(), L.c.done, sizeof(int) * L.k, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        L.active = 0;
        bool all_final = true;
        for (int j = 0; j < L.k; ++j) {
            if (!L.fin[j] && mask[i * KMAX + j] && done[j]) {  // re-arming found nothing to do
                L.fin[j] = 1;
                L.fstat[j] = L.rel[j] <= s->opt.tol ? GB_OK : GB_BREAKDOWN;
            }
            if (!L.fin[j]) { all_final = false; L.active += done[j] ? 0 : 1; }
        }
        if (all_final) {
            int st2 = GB_OK;
            for (int j = 0; j < L.k; ++j) if (L.fstat[j] != GB_OK) st2 = L.fstat[j];
            retire(s, L, st2);
        } else {
            L.state = L.active ? SL_ITER : SL_SERVICE;
        }
    }
    return GB_OK;
}

// ------------------------------------------------------ persistent lane --
// One launch per tier over every slot of that tier waiting for it (their
// initial residuals formed at admission, which synchronised its stream), each
// on a stream of its own.
static int launch_persistent_tier(gb_server *s, int tier);
static int launch_persistent(gb_server *s) {
    GB_TRY(launch_persistent_tier(s, 1));
    return launch_persistent_tier(s, 2);
}
static int launch_persistent_tier(gb_server *s, int tier) {
    std::vector<Slot *> w;
    for (auto &p : s->slots) if (p->state == SL_PWAIT && p->ptier == tier) w.push_back(p.get());
    if (w.empty()) return GB_OK;
    const bool ru = s->opt.precision != GB_F64;
    auto L = std::make_unique<gb_server::PLaunch>();
    GB_CHECK_CUDA(cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking));
    cudaStream_t st = L->st;
    const int m = (int)w.size();
    std::vector<BSys> tab;
    std::vector<int> list(m + 1, 0);  // list, then the block counter
    long long maxit = 1;
    for (int i = 0; i < m; ++i) {
        tab.push_back(desc_of(*w[i], 0));
        list[i] = i;
        maxit = std::max<long long>(maxit, 20 * (long long)w[i]->n + 100);
    }
    GB_CHECK_CUDA(cudaMallocAsync((void **)&L->d_tab, sizeof(BSys) * m, st));
    GB_CHECK_CUDA(cudaMallocAsync((void **)&L->d_list, sizeof(int) * (m + 1), st));
    GB_CHECK_CUDA(cudaMemcpyAsync(L->d_tab, tab.data(), sizeof(BSys) * m, cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemcpyAsync(L->d_list, list.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, st));
    PersistOpts po{};
    po.tol = s->opt.tol;
    po.inner_tol = 1e-4;
    po.maxit = std::min<long long>(s->opt.max_iter, maxit);
    po.max_outer = ru ? 30 : 50;
    ::gb::count_launches(1);
    if (tier == 2) {
        const int grid = std::min(m, std::max(1, num_sms() / CLUSTER_CS)) * CLUSTER_CS;
        if (ru) k_bcluster<float><<<grid, PNT, 0, st>>>(L->d_tab, L->d_list, m, L->d_list + m, po);
        else k_bcluster<double><<<grid, PNT, 0, st>>>(L->d_tab, L->d_list, m, L->d_list + m, po);
    } else {
        const int grid = std::min(m, num_sms() * 2);
        if (ru) k_bpersist<float><<<grid, PNT, 0, st>>>(L->d_tab, L->d_list, m, L->d_list + m, po);
        else k_bpersist<double><<<grid, PNT, 0, st>>>(L->d_tab, L->d_list, m, L->d_list + m, po);
    }
    GB_CHECK_CUDA(cudaGetLastError());
    GB_CHECK_CUDA(cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming));
    GB_CHECK_CUDA(cudaEventRecord(L->done, st));
    for (Slot *x : w) x->state = SL_PRUN;
    L->slots = std::move(w);
    s->plaunch.push_back(std::move(L));
    return GB_OK;
}

// Finished persistent launches: converged columns are final; any other column
// is re-armed with a fresh direction by the service step and goes on in the
// lock-step loop from the current x.  Returns whether one finished.
static int poll_persistent(gb_server *s, bool *finished) {
    *finished = false;
    const bool ru = s->opt.precision != GB_F64;
    for (size_t li = 0; li < s->plaunch.size();) {
        auto &L = s->plaunch[li];
        const cudaError_t q = cudaEventQuery(L->done);
        if (q == cudaErrorNotReady) { ++li; continue; }
        GB_CHECK_CUDA(q);
        for (Slot *x : L->slots) {
            Slot &S = *x;
            std::vector<double> rr(S.k), bb(S.k);
            GB_CHECK_CUDA(cudaMemcpy(rr.data(), S.c.rr, sizeof(double) * S.k, cudaMemcpyDeviceToHost));
            GB_CHECK_CUDA(cudaMemcpy(bb.data(), S.c.bb, sizeof(double) * S.k, cudaMemcpyDeviceToHost));
            std::vector<int> rearm(S.k, 0);
            std::vector<long long> it0(S.k, 0);
            bool left = false;
            for (int j = 0; j < S.k; ++j) {
                if (S.fin[j]) continue;
                S.rel[j] = bb[j] > 0 ? std::sqrt(rr[j] / bb[j]) : 0.0;
                if (S.rel[j] <= s->opt.tol) { S.fin[j] = 1; S.fstat[j] = GB_OK; }
                else { rearm[j] = ST_BREAK; left = true; }  // the service step re-arms it with a fresh direction
            }
            if (left) {
                GB_CHECK_CUDA(cudaMemcpy(S.c.status, rearm.data(), sizeof(int) * S.k, cudaMemcpyHostToDevice));
                GB_CHECK_CUDA(cudaMemcpy(S.c.it, it0.data(), sizeof(long long) * S.k, cudaMemcpyHostToDevice));
                if (ru) GB_CHECK_CUDA(cudaMemset(S.X, 0, sizeof(float) * (size_t)S.n * S.k));  // its correction is in X64
            }
            S.active = 0;
            S.state = SL_SERVICE;
        }
        cudaFreeAsync(L->d_tab, L->st);
        cudaFreeAsync(L->d_list, L->st);
        cudaEventDestroy(L->done);
        cudaStreamDestroy(L->st);
        s->plaunch.erase(s->plaunch.begin() + li);
        *finished = true;
    }
    return GB_OK;
}

// ---------------------------------------------------------------- loop --
static void server_loop(gb_server *s) {
    cudaSetDevice(s->dev);
    const bool ru = s->opt.precision != GB_F64;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            while (!s->inbox.empty()) { s->pending.push_back(std::move(s->inbox.front())); s->inbox.pop_front(); }
            if (s->stopping && s->pending.empty() && s->slots.empty()) break;
            if (s->pending.empty() && s->slots.empty()) {
                s->cv.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
        }
        // A. launch a chunk of CG iterations for the iterating slots of each
        // lane (the lane's stream; the two lanes' chunks run side by side)
        gb::Range round_range("gbpcg:serve_round");
        std::vector<Slot *> lane_slots[gb_server::NLANES];
        for (auto &p : s->slots) if (p->state == SL_ITER) lane_slots[p->lane].push_back(p.get());
        bool launched[gb_server::NLANES] = {};
        for (int li = 0; li < gb_server::NLANES && s->fatal == GB_OK; ++li) {
            std::vector<Slot *> &it_slots = lane_slots[li];
            gb_server::Lane &Ln = s->ln[li];
            if (it_slots.empty()) continue;
            // the table in width-class order: each class's units are contiguous
            std::stable_sort(it_slots.begin(), it_slots.end(),
                             [](const Slot *a, const Slot *b) { return width_class(a->k) < width_class(b->k); });
            std::vector<BSys> tab;
            std::vector<int> umap;
            ClassRanges cls;
            for (int c = 0; c < ClassRanges::N; ++c) cls.base[c] = -1;
            for (size_t i = 0; i < it_slots.size(); ++i) {
                const int c = width_class(it_slots[i]->k);
                if (cls.base[c] < 0) cls.base[c] = (int)umap.size();
                tab.push_back(desc_of(*it_slots[i], (int)umap.size()));
                for (int u = 0; u < it_slots[i]->units; ++u) umap.push_back((int)i);
                cls.count[c] = (int)umap.size() - cls.base[c];
            }
            for (int c = 0; c < ClassRanges::N; ++c) if (cls.base[c] < 0) cls.base[c] = 0;
            int rc = grow(s, &Ln.d_unit_sys, &Ln.cap_umap, umap.size(), Ln.st);
            if (rc == GB_OK) rc = grow(s, &Ln.d_partials, &Ln.cap_part, umap.size() * 3 * KMAX, Ln.st);
            BGlobal g{};
            g.maxit = s->opt.max_iter;
            g.active_systems = (int)it_slots.size();
            g.stop_on_retire = 1;
            const bool adaptive = s->opt.iters_per_step <= 0;
            const int ips = adaptive ? Ln.ips : s->opt.iters_per_step;
            g.budget = ips;
            cudaError_t e = cudaMemcpyAsync(Ln.d_sys, tab.data(), sizeof(BSys) * tab.size(), cudaMemcpyHostToDevice, Ln.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(Ln.d_unit_sys, umap.data(), sizeof(int) * umap.size(), cudaMemcpyHostToDevice, Ln.st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(Ln.d_G, &g, sizeof(g), cudaMemcpyHostToDevice, Ln.st);
            const int U = (int)umap.size();
            if (e == cudaSuccess && adaptive) e = cudaEventRecord(Ln.ev0, Ln.st);
            for (int i = 0; i < ips && e == cudaSuccess && rc == GB_OK; ++i) {
                ::gb::count_launches(2);
                if (ru) {
                    launch_bspmm<float, float>(true, cls, U, Ln.d_sys, Ln.d_unit_sys, Ln.d_G, Ln.d_partials, Ln.st);
                    k_bupdate<float><<<U, NT, 0, Ln.st>>>(Ln.d_sys, Ln.d_unit_sys, Ln.d_G, Ln.d_partials);
                    k_bpupdate<float><<<U, NT, 0, Ln.st>>>(Ln.d_sys, Ln.d_unit_sys, Ln.d_G);
                } else {
                    launch_bspmm<double, double>(true, cls, U, Ln.d_sys, Ln.d_unit_sys, Ln.d_G, Ln.d_partials, Ln.st);
                    k_bupdate<double><<<U, NT, 0, Ln.st>>>(Ln.d_sys, Ln.d_unit_sys, Ln.d_G, Ln.d_partials);
                    k_bpupdate<double><<<U, NT, 0, Ln.st>>>(Ln.d_sys, Ln.d_unit_sys, Ln.d_G);
                }
            }
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess && adaptive) e = cudaEventRecord(Ln.ev1, Ln.st);
            if (e == cudaSuccess) e = cudaEventRecord(Ln.ev, Ln.st);
            if (e != cudaSuccess || rc != GB_OK) {
                s->fatal = e != cudaSuccess ? GB_ECUDA : rc;
                s->fatal_msg = e != cudaSuccess ? cudaGetErrorString(e) : gbpcg_last_error();
                break;
            }
            launched[li] = true;
            s->stats.steps += 1;
        }
        if (s->fatal != GB_OK) break;
        // B. admit while the chunk runs (side stream)
        while (!s->pending.empty() && (int)s->slots.size() < s->opt.max_slots) {
            SReq &q = s->pending.front();
            const size_t est = estimate_bytes(q.r, ru);
            if (est > s->opt.mem_budget) {
                set_error("request %llu needs ~%zu bytes, above the budget", (unsigned long long)q.ticket, est);
                finish(s, q, GB_TOO_LARGE, nullptr);
                s->pending.pop_front();
                continue;
            }
            if (s->in_use + est > s->opt.mem_budget) break;  // wait for memory
            std::unique_ptr<Slot> sl;
            const int rc = admit(s, q, sl);
            if (rc != GB_OK) {
                finish(s, q, rc, nullptr);
                s->pending.pop_front();
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->stats.resident += 1;
                s->stats.max_resident = std::max<int32_t>(s->stats.max_resident, (int32_t)s->stats.resident);
            }
            s->slots.push_back(std::move(sl));
            s->pending.pop_front();
        }
        // B'. one persistent launch for the requests admitted to that lane
        {
            const int rc = launch_persistent(s);
            if (rc != GB_OK) { s->fatal = rc; s->fatal_msg = gbpcg_last_error(); break; }
        }
        // C. wait for each lane's chunk, pull the column states of its slots
        for (int li = 0; li < gb_server::NLANES && s->fatal == GB_OK; ++li) {
            if (!launched[li]) continue;
            gb_server::Lane &Ln = s->ln[li];
            cudaError_t e = cudaEventSynchronize(Ln.ev);
            if (e == cudaSuccess && s->opt.iters_per_step <= 0) {
                // adaptive chunk length: about CHUNK_MS of iterations of the
                // lane's resident set per chunk, so that arrivals are admitted
                // (and small requests solved) within about that long
                BGlobal hg{};
                float ms = 0.f;
                e = cudaMemcpy(&hg, Ln.d_G, sizeof(hg), cudaMemcpyDeviceToHost);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, Ln.ev0, Ln.ev1);
                const int done_its = std::max(1, Ln.ips - std::max(0, hg.budget));
                if (e == cudaSuccess && ms > 0.f) {
                    const double per_it = (double)ms / done_its;
                    const double want = CHUNK_MS / std::max(per_it, 1e-3);
                    Ln.ips = (int)std::max(4.0, std::min(200.0, want));
                }
            }
            for (Slot *L : lane_slots[li]) {
                if (e != cudaSuccess) break;
                std::vector<int> done(L->k);
                e = cudaMemcpy(done.data(), L->c.done, sizeof(int) * L->k, cudaMemcpyDeviceToHost);
                int a = 0;
                for (int j = 0; j < L->k; ++j) a += (!L->fin[j] && !done[j]) ? 1 : 0;
                L->active = a;
                if (a == 0) L->state = SL_SERVICE;
            }
            if (e != cudaSuccess) { s->fatal = GB_ECUDA; s->fatal_msg = cudaGetErrorString(e); }
        }
        if (s->fatal != GB_OK) break;
        const bool any_launched = launched[0] || launched[1];
        // C'. persistent launches that have finished
        bool pdone = false;
        {
            const int rc = poll_persistent(s, &pdone);
            if (rc != GB_OK) { s->fatal = rc; s->fatal_msg = gbpcg_last_error(); break; }
        }
        if (!any_launched && !pdone && !s->plaunch.empty()) {
            // only persistent launches in flight: poll them gently
            bool serviceable = false;
            for (auto &p : s->slots) serviceable |= p->state == SL_SERVICE;
            if (!serviceable) std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
        // D. service slots whose columns all stopped; E. drop retired slots
        std::vector<Slot *> sv;
        for (auto &p : s->slots) if (p->state == SL_SERVICE) sv.push_back(p.get());
        const int rc = service(s, sv);
        if (rc != GB_OK) { s->fatal = rc; s->fatal_msg = gbpcg_last_error(); break; }
        s->slots.erase(std::remove_if(s->slots.begin(), s->slots.end(),
                                      [](const std::unique_ptr<Slot> &p) { return p->state == SL_DONE; }),
                       s->slots.end());
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stats.mem_in_use = (double)s->in_use;
            s->stats.mem_peak = (double)s->peak;
        }
    }
    // fatal error or stop: fail whatever is left (after any persistent launch
    // still using the slots' buffers has finished)
    for (auto &Ln : s->ln) cudaStreamSynchronize(Ln.st);
    for (auto &L : s->plaunch) {
        cudaStreamSynchronize(L->st);
        cudaFreeAsync(L->d_tab, L->st);
        cudaFreeAsync(L->d_list, L->st);
        cudaEventDestroy(L->done);
        cudaStreamDestroy(L->st);
    }
    s->plaunch.clear();
    for (auto &p : s->slots) { finish(s, p->q, s->fatal ? s->fatal : GB_EINVAL, p.get()); release_slot(s, *p); }
    s->slots.clear();
    for (auto &q : s->pending) finish(s, q, s->fatal ? s->fatal : GB_EINVAL, nullptr);
    s->pending.clear();
    cudaStreamSynchronize(s->side_st);
    for (auto &Ln : s->ln) cudaStreamSynchronize(Ln.st);
}

// ================================================================= ABI ==
// Releases what serve_create made of a server whose thread never started.
static void release_unstarted(gb_server *s) {
    for (auto &Ln : s->ln) {
        cudaFree(Ln.d_sys); cudaFree(Ln.d_G);
        if (Ln.ev) cudaEventDestroy(Ln.ev);
        if (Ln.ev0) cudaEventDestroy(Ln.ev0);
        if (Ln.ev1) cudaEventDestroy(Ln.ev1);
        if (Ln.st) cudaStreamDestroy(Ln.st);
    }
    cudaFree(s->d_mask); cudaFree(s->d_sys1); cudaFree(s->d_mask1);
    if (s->side_st) cudaStreamDestroy(s->side_st);
    delete s;
}

extern "C" int serve_create(const ServeOptions *opt, const gb_allocator *alloc, gb_server **out) {
    GB_REQUIRE(opt && out, "serve_create: NULL argument");
    *out = nullptr;
    GB_REQUIRE(opt->mem_budget >= (1u << 20), "serve_create: mem_budget below 1 MB");
    GB_REQUIRE(opt->max_slots >= 1 && opt->max_slots <= 4096, "serve_create: max_slots not in 1..4096");
    GB_REQUIRE(opt->precision == GB_F64 || opt->precision == GB_F32_RU,
               "serve_create: precision must be GB_F64 or GB_F32_RU");
    GB_REQUIRE(!alloc || (alloc->alloc && alloc->free), "serve_create: allocator without alloc/free");
    int prev = 0;
    GB_CHECK_CUDA(cudaGetDevice(&prev));
    gb_server *s = new gb_server();
    s->opt = *opt;
    if (alloc) s->user = *alloc;
    if (!(s->opt.tol > 0)) s->opt.tol = 1e-10;
    if (s->opt.max_iter <= 0) s->opt.max_iter = 1000000;
    if (s->opt.iters_per_step < 0) s->opt.iters_per_step = 0;
    s->alloc.ctx = s;
    s->alloc.alloc = srv_alloc;
    s->alloc.free = srv_free;
    const char *what = nullptr;
    cudaError_t e = cudaSuccess;
#define GB_SC(expr) if (e == cudaSuccess && (e = (expr)) != cudaSuccess) what = #expr
    if (opt->device >= 0) GB_SC(cudaSetDevice(opt->device));
    GB_SC(cudaGetDevice(&s->dev));
    for (int li = 0; li < gb_server::NLANES; ++li) {
        gb_server::Lane &Ln = s->ln[li];
        GB_SC(cudaStreamCreateWithFlags(&Ln.st, cudaStreamNonBlocking));
        GB_SC(cudaEventCreateWithFlags(&Ln.ev, cudaEventDisableTiming));
        GB_SC(cudaEventCreate(&Ln.ev0));
        GB_SC(cudaEventCreate(&Ln.ev1));
        GB_SC(cudaMalloc((void **)&Ln.d_sys, sizeof(BSys) * s->opt.max_slots));
        GB_SC(cudaMalloc((void **)&Ln.d_G, sizeof(BGlobal)));
    }
    GB_SC(cudaStreamCreateWithFlags(&s->side_st, cudaStreamNonBlocking));
    GB_SC(cudaMalloc((void **)&s->d_mask, sizeof(int) * KMAX * s->opt.max_slots));
    GB_SC(cudaMalloc((void **)&s->d_sys1, sizeof(BSys)));
    GB_SC(cudaMalloc((void **)&s->d_mask1, sizeof(int) * KMAX));
#undef GB_SC
    if (e != cudaSuccess) {
        set_error("serve_create: %s: %s", what, cudaGetErrorString(e));
        release_unstarted(s);
        cudaSetDevice(prev);
        return e == cudaErrorMemoryAllocation ? GB_ENOMEM : GB_ECUDA;
    }
    s->th = std::thread(server_loop, s);
    cudaSetDevice(prev);
    *out = s;
    return GB_OK;
}

extern "C" int serve_submit(gb_server *s, const ServeRequest *r, uint64_t *ticket) {
    GB_REQUIRE(s && r && ticket, "serve_submit: NULL argument");
    GB_REQUIRE(r->k >= 1 && r->k <= KMAX, "serve_submit: k must be in 1..%d", KMAX);
    GB_REQUIRE(r->h_x, "serve_submit: h_x (result buffer) is NULL");
    GB_REQUIRE(r->h_gB || (r->gid >= 0 && r->gid <= 4), "serve_submit: need h_gB or a Dirichlet id 0..4");
    SReq q;
    q.r = *r;
    const int nc = r->gid == 3 ? 4 : (r->gid == 4 ? 10 : 0);
    if (!r->h_gB && nc) {
        GB_REQUIRE(r->h_coef, "serve_submit: Dirichlet id %d needs coefficients", r->gid);
        q.coef.assign(r->h_coef, r->h_coef + (size_t)nc * r->k);
    }
    q.t_submit = now_ms();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) { set_error("serve_submit: server is shutting down"); return GB_EINVAL; }
    if (s->fatal) { set_error("serve_submit: server stopped after an error: %s", s->fatal_msg.c_str()); return s->fatal; }
    q.ticket = s->next_ticket++;
    *ticket = q.ticket;
    s->inbox.push_back(std::move(q));
    s->stats.submitted += 1;
    s->cv.notify_one();
    return GB_OK;
}

extern "C" int serve_poll(gb_server *s, uint64_t ticket, ServeResult *out) {
    GB_REQUIRE(s && out, "serve_poll: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) {
        if (ticket == 0 || ticket >= s->next_ticket) { set_error("serve_poll: unknown ticket %llu", (unsigned long long)ticket); return GB_EINVAL; }
        return GB_PENDING;
    }
    *out = it->second;
    s->results.erase(it);
    return out->status;
}

extern "C" int serve_stats(gb_server *s, ServeStats *out) {
    GB_REQUIRE(s && out, "serve_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->pending = (int64_t)(s->stats.submitted - s->stats.completed - s->stats.resident);
    return GB_OK;
}

extern "C" void serve_destroy(gb_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (auto &Ln : s->ln) {
        cudaFree(Ln.d_sys); cudaFree(Ln.d_unit_sys); cudaFree(Ln.d_G); cudaFree(Ln.d_partials);
        cudaEventDestroy(Ln.ev);
        cudaEventDestroy(Ln.ev0);
        cudaEventDestroy(Ln.ev1);
        cudaStreamDestroy(Ln.st);
    }
    cudaFree(s->d_mask);
    cudaFree(s->d_sys1); cudaFree(s->d_unit1); cudaFree(s->d_mask1); cudaFree(s->d_partials1);
    cudaStreamDestroy(s->side_st);
    delete s;
}
