// batched.cu -- pcg_solve_batched: many systems, each with k <= 32 right-hand
// sides (Eq. MRH of Sec. 4.3, "block of r.h.s. terms"), solved by k
// independent Jacobi-PCG recurrences per system that share one SELL pass per
// iteration (SpMM), all systems advancing in the same three launches.
//
// Work decomposition: every system is cut into "units" of consecutive rows;
// one block owns one unit.  Inside a block, threads form groups of kw lanes
// (kw = the power of two >= k): a group owns one row and lane j owns column j,
// so the k values of a row-major block row are read and written together.
// Each unit writes per-column partial sums; the last block of a system (per-
// system ticket) reduces them in unit order -- deterministic -- and updates
// that system's per-column scalars.  A column that meets Eq. (2) is frozen
// (convergence mask); a system whose columns are all frozen leaves the loop,
// and the block that retires the last system clears the while-node condition.
//
// precision GB_F64 runs the recurrences in fp64; GB_F32_IR / GB_BF16_IR wrap
// fp32 recurrences (fp32 or bf16 values) in fp64 iterative refinement: outer
// residual B - A X, convergence test and update X += ||r_j|| D_j in fp64;
// GB_F32_RU keeps one fp32 recurrence per column and makes fp64 reliable
// updates (X += D, R = B - A X, residual replacement) every 10x decrease.
#include <map>

#include "batched.cuh"


using namespace gb;

template <class TV>
static int batched_ir(Batch &b, const PcgOptions &o, cudaStream_t st, std::vector<int> &outer_cnt,
                      std::vector<long long> &inner_its) {
    const size_t ns = b.h.size();
    HostCols hc;
    std::vector<int> mask(ns * KMAX, 0);
    std::vector<double> prev;
    // (outer_cnt / inner_its: zero on entry, or the persistent tiers' counts)
    // scale = ||r_j|| kept in c.scale; the fp32 recurrence works on R/||r||
    for (int outer = 0; outer < o.max_outer; ++outer) {
        GB_TRY(pull_cols(b, hc, st));
        bool any = false;
        std::vector<double> scale;
        for (size_t s = 0; s < ns; ++s) {
            const int k = b.h[s].k;
            scale.assign(k, 1.0);
            for (int j = 0; j < k; ++j) {
                const bool need = hc.bb[s][j] > 0 && hc.rr[s][j] > o.tol * o.tol * hc.bb[s][j];
                mask[s * KMAX + j] = need ? 1 : 0;
                scale[j] = need ? std::sqrt(hc.rr[s][j]) : 1.0;
                any |= need;
                if (need) outer_cnt[s] += 1;
            }
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.scale, scale.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
            // inner threshold: ||r32|| = 1, stop at inner_tol
            std::vector<double> th(k, o.inner_tol * o.inner_tol);
            std::vector<long long> z(k, 0);
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.thresh, th.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.it, z.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, st));
            GB_CHECK_CUDA(cudaStreamSynchronize(st));
        }
        if (!any) break;
        GB_CHECK_CUDA(cudaMemcpyAsync(b.d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
        ::gb::count_launches(1); k_bscale_down<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_mask);
        GB_TRY((start_and_loop<float, TV>(b, mask, o.max_iter, o, st)));
        HostCols hi;
        GB_TRY(pull_cols(b, hi, st));
        for (size_t s = 0; s < ns; ++s) {
            long long mx = 0;
            for (int j = 0; j < b.h[s].k; ++j) if (mask[s * KMAX + j]) mx = std::max(mx, hi.it[s][j]);
            inner_its[s] += mx;
        }
        ::gb::count_launches(1); k_bcorrect<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_mask);
        ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 0, 0, o.tol);
        GB_CHECK_CUDA(cudaGetLastError());
        // restore the outer thresholds (tol^2 ||b||^2) for the next test
        for (size_t s = 0; s < ns; ++s) {
            std::vector<double> th(b.h[s].k);
            for (int j = 0; j < b.h[s].k; ++j) th[j] = o.tol * o.tol * hc.bb[s][j];
            GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.thresh, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, st));
        }
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
    }
    return GB_OK;
}

// fp32 recurrences with fp64 reliable updates (GB_F32_RU): every column's
// fp32 recurrence runs on the unscaled residual until it has fallen by a
// factor 10 (threshold max(0.01 ||r||^2, target), target = (tol/2)^2 ||b||^2);
// then, for the columns that ran, X += D in fp64 (k_bcorrect), the true
// residual R = B - A X in fp64 (k_bresid), and the test of Eq. 2.  A column
// above tol goes on with its fp32 residual replaced by the true one and its
// direction kept (k_breplace / k_breplace_p: mask 1), or restarted with a
// fresh direction after a breakdown (mask 2); four updates in a row without
// a 10 % gain, or the iteration cap, stop it (the fp64 finish of the caller
// then takes it from its X).  The Krylov recurrence is not restarted at each
// update, so the iteration count stays close to the fp64 recurrence's,
// unlike iterative refinement's restarted inner solves.
template <class TV>
static int batched_ru(Batch &b, const PcgOptions &o, cudaStream_t st, std::vector<int> &updates,
                      std::vector<long long> &its) {
    const size_t ns = b.h.size();
    HostCols hc;
    GB_TRY(pull_cols(b, hc, st));
    std::vector<int> mask(ns * KMAX, 0);
    std::vector<std::vector<double>> best(ns);
    std::vector<std::vector<int>> stalls(ns), fin(ns);
    bool any = false;  // (updates / its: zero on entry, or the persistent tiers' counts)
    for (size_t s = 0; s < ns; ++s) {
        const int k = b.h[s].k;
        best[s].assign(k, 1.0);
        stalls[s].assign(k, 0);
        fin[s].assign(k, 0);
        std::vector<double> target(k), one(k, 1.0);
        for (int j = 0; j < k; ++j) {
            target[j] = 0.25 * o.tol * o.tol * hc.bb[s][j];
            const bool need = hc.bb[s][j] > 0 && hc.rr[s][j] > o.tol * o.tol * hc.bb[s][j];
            mask[s * KMAX + j] = need ? 2 : 0;
            fin[s][j] = need ? 0 : 1;
            any |= need;
        }
        GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.target, target.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.scale, one.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        std::vector<long long> z(k, 0);
        GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.it, z.data(), sizeof(long long) * k, cudaMemcpyHostToDevice, st));
    }
    std::vector<BSys> hs(ns);
    while (any) {
        GB_CHECK_CUDA(cudaMemcpyAsync(b.d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
        ::gb::count_launches(2);
        k_breplace<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, b.d_mask, 0.01);
        k_breplace_p<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_mask);
        GB_CHECK_CUDA(cudaGetLastError());
        GB_CHECK_CUDA(cudaMemcpyAsync(hs.data(), b.d_sys, sizeof(BSys) * ns, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        int act = 0;
        for (auto &x : hs) act += x.active > 0 ? 1 : 0;
        if (act > 0) {
            BGlobal g{};
            g.maxit = o.max_iter;
            g.active_systems = act;
            g.budget = -1;
            GB_CHECK_CUDA(cudaMemcpyAsync(b.d_G, &g, sizeof(g), cudaMemcpyHostToDevice, st));
            GB_TRY(run_bloop(st, b.d_G, o.use_graph != 0, o.check_every,
                             [&](cudaStream_t s2) { enqueue_biter<float, TV>(b, s2); }));
        }
        // reliable update of the columns that ran: X += D, R = B - A X (fp64)
        ::gb::count_launches(2);
        k_bcorrect<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_mask);
        k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 0, 0, o.tol);
        GB_CHECK_CUDA(cudaGetLastError());
        GB_TRY(pull_cols(b, hc, st));
        any = false;
        for (size_t s = 0; s < ns; ++s) {
            bool ran = false;
            for (int j = 0; j < b.h[s].k; ++j) {
                int &m = mask[s * KMAX + j];
                if (!m) continue;
                ran = true;
                its[s] = std::max(its[s], hc.it[s][j]);
                const double rel = hc.bb[s][j] > 0 ? std::sqrt(hc.rr[s][j] / hc.bb[s][j]) : 0.0;
                int nm = 0;
                if (rel <= o.tol || hc.status[s][j] == ST_MAXIT || hc.it[s][j] >= o.max_iter) {
                    fin[s][j] = 1;
                } else {
                    if (rel < 0.9 * best[s][j]) { best[s][j] = rel; stalls[s][j] = 0; }
                    else if (++stalls[s][j] >= 4) fin[s][j] = 1;
                    if (!fin[s][j]) nm = hc.status[s][j] == ST_BREAK ? 2 : 1;
                }
                m = nm;
                any |= nm != 0;
            }
            if (ran) updates[s] += 1;
        }
    }
    return GB_OK;
}

// Builds the batch: per-system units, permuted fp64 right-hand sides and
// starting iterates, recurrence vectors of the precision's type, column state,
// and the device copies of the system table.
static int setup_batch(Batch &b, int nsys, const gb_sell *const *A, const double *const *d_B,
                       double *const *d_X, const int *k, const PcgOptions &o, cudaStream_t st) {
    const bool ir = o.precision != GB_F64;
    b.mem = Mem(nullptr, st);
    b.h.resize(nsys);
    b.tma = true;
    for (int s = 0; s < nsys; ++s) b.tma = b.tma && A[s]->C == 32;
    // unit table: systems in width-class order (a class's units contiguous)
    std::vector<int> unit_sys;
    b.cls = ClassRanges{};
    for (int c = 0; c < ClassRanges::N; ++c) {
        b.cls.base[c] = (int)unit_sys.size();
        for (int s = 0; s < nsys; ++s) {
            if (width_class(k[s]) != c) continue;
            BSys &S = b.h[s];
            S.unit0 = (int)unit_sys.size();
            S.nunits = units_of_rows(A[s]->n, &S.rows_per_unit);
            for (int u = 0; u < S.nunits; ++u) unit_sys.push_back(s);
        }
        b.cls.count[c] = (int)unit_sys.size() - b.cls.base[c];
    }
    for (int s = 0; s < nsys; ++s) {
        BSys &S = b.h[s];
        const gb_sell *M = A[s];
        const int64_t n = M->n;
        const int unit0 = S.unit0, nunits = S.nunits;
        const int64_t rpu = S.rows_per_unit;
        S = BSys{};
        S.A = M->view();
        S.k = k[s];
        S.kw = kw_of(k[s]);
        S.unit0 = unit0;
        S.nunits = nunits;
        S.rows_per_unit = rpu;
        const size_t nk = (size_t)n * S.k;
        double *B64, *X64, *R64;
        GB_TRY(b.take(&B64, nk));
        GB_TRY(b.take(&X64, nk));
        GB_TRY(b.take(&R64, nk));
        S.B64 = B64; S.X64 = X64; S.R64 = R64;
        if (!ir) {
            double *P, *Q;
            GB_TRY(b.take(&P, nk));
            GB_TRY(b.take(&Q, nk));
            S.X = X64; S.R = R64; S.P = P; S.Q = Q;
            S.val = M->val;
        } else {
            float *X, *R, *P, *Q;
            GB_TRY(b.take(&X, nk));
            GB_TRY(b.take(&R, nk));
            GB_TRY(b.take(&P, nk));
            GB_TRY(b.take(&Q, nk));
            S.X = X; S.R = R; S.P = P; S.Q = Q;
            S.val = o.precision == GB_BF16_IR ? (const void *)M->val16 : (const void *)M->val32;
        }
        double *cd;
        GB_TRY(b.take(&cd, (size_t)10 * KMAX));
        S.c.rho = cd; S.c.pq = cd + KMAX; S.c.alpha = cd + 2 * KMAX; S.c.beta = cd + 3 * KMAX;
        S.c.rr = cd + 4 * KMAX; S.c.bb = cd + 5 * KMAX; S.c.thresh = cd + 6 * KMAX; S.c.scale = cd + 7 * KMAX;
        S.c.pz = cd + 8 * KMAX; S.c.target = cd + 9 * KMAX;
        long long *ci;
        GB_TRY(b.take(&ci, (size_t)KMAX));
        S.c.it = ci;
        int *cs;
        GB_TRY(b.take(&cs, (size_t)2 * KMAX));
        S.c.done = cs; S.c.status = cs + KMAX;
        GB_CHECK_CUDA(cudaMemsetAsync(cd, 0, sizeof(double) * 10 * KMAX, st));
        GB_CHECK_CUDA(cudaMemsetAsync(ci, 0, sizeof(long long) * KMAX, st));
        GB_CHECK_CUDA(cudaMemsetAsync(cs, 0, sizeof(int) * 2 * KMAX, st));
        const int g = stride_grid((int64_t)nk, 256, 8);
        ::gb::count_launches(1); k_gather_rows<<<g, 256, 0, st>>>(n, S.k, M->perm, d_B[s], B64);
        ::gb::count_launches(1); k_gather_rows<<<g, 256, 0, st>>>(n, S.k, M->perm, (o.x0_zero || !d_X) ? nullptr : d_X[s], X64);
    }
    b.units = (int)unit_sys.size();
    GB_TRY(b.take(&b.d_sys, (size_t)nsys));
    GB_TRY(b.take(&b.d_unit_sys, unit_sys.size()));
    GB_TRY(b.take(&b.d_mask, (size_t)nsys * KMAX));
    GB_TRY(b.take(&b.d_G, 1));
    GB_TRY(b.take(&b.partials, (size_t)b.units * 3 * KMAX));
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_sys, b.h.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_unit_sys, unit_sys.data(), sizeof(int) * unit_sys.size(), cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemsetAsync(b.d_G, 0, sizeof(BGlobal), st));

    return GB_OK;
}

// One launch of a persistent kernel over the systems in `list` (their
// initial residuals already formed): fp64 CG for fp64 batches, fp32 correction
// solves in fp64 refinement otherwise.  tier 1: one block per system
// (k_bpersist); tier 2: one cluster of CLUSTER_CS blocks per system
// (k_bcluster), as many clusters as the SMs hold side by side; tier 3: one
// group of G blocks per system (k_bgrid, a cooperative launch), as many
// groups as the device holds.  Returns 1 when tier 3 cannot be resident.
static int run_persist(Batch &b, const std::vector<int> &list, const PcgOptions &o, bool ir, cudaStream_t st,
                       int tier = 1) {
    int *d_list = nullptr, *d_next = nullptr;
    GB_TRY(b.take(&d_list, list.size()));
    GB_TRY(b.take(&d_next, 1));
    GB_CHECK_CUDA(cudaMemcpyAsync(d_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaMemsetAsync(d_next, 0, sizeof(int), st));
    PersistOpts po{};
    po.tol = o.tol;
    po.inner_tol = ir ? std::min(o.inner_tol, 1e-4) : 0.0;
    po.maxit = o.max_iter;
    po.max_outer = ir ? o.max_outer : 50;
    if (tier == 3) {
        // `list` holds systems of one group size G (the caller buckets them):
        // groups of G blocks of one cooperative launch
        const int res = ir ? grid_resident_blocks<float>() : grid_resident_blocks<double>();
        if (res <= 0) return 1;
        const int G = grid_blocks_for(b.h[list[0]].A.n, kw_of(b.h[list[0]].k), res);
        const int groups = (int)std::min<size_t>(list.size(), (size_t)std::max(1, res / G));
        char *ws = nullptr;
        const size_t wb = grid_ws_bytes(groups, G);
        GB_TRY(b.take(&ws, wb));
        GB_CHECK_CUDA(cudaMemsetAsync(ws, 0, wb, st));
        int *d_err = nullptr;
        if (ir) GB_TRY(launch_grid<float>(b.d_sys, d_list, (int)list.size(), d_next, G, groups, ws, po, st, &d_err));
        else GB_TRY(launch_grid<double>(b.d_sys, d_list, (int)list.size(), d_next, G, groups, ws, po, st, &d_err));
        b.grid_err.push_back(d_err);
        return GB_OK;
    }
    ::gb::count_launches(1);
    if (tier == 2) {
        const int nclu = (int)std::min<size_t>(list.size(), (size_t)std::max(1, num_sms() / CLUSTER_CS));
        if (ir) k_bcluster<float><<<nclu * CLUSTER_CS, PNT, 0, st>>>(b.d_sys, d_list, (int)list.size(), d_next, po);
        else k_bcluster<double><<<nclu * CLUSTER_CS, PNT, 0, st>>>(b.d_sys, d_list, (int)list.size(), d_next, po);
    } else {
        const int grid = (int)std::min<size_t>(list.size(), (size_t)num_sms() * 2);
        if (ir) k_bpersist<float><<<grid, PNT, 0, st>>>(b.d_sys, d_list, (int)list.size(), d_next, po);
        else k_bpersist<double><<<grid, PNT, 0, st>>>(b.d_sys, d_list, (int)list.size(), d_next, po);
    }
    GB_CHECK_CUDA(cudaGetLastError());
    return GB_OK;
}

extern "C" int pcg_solve_batched(int nsys, const gb_sell *const *A, const double *const *d_B,
                                 double *const *d_X, const int *k, const PcgOptions *opt, void *stream,
                                 PcgStats *stats) {
    gb::Range range("gbpcg:pcg_solve_batched");
    GB_REQUIRE(nsys >= 1 && A && d_B && d_X && k && stats, "pcg_solve_batched: NULL argument");
    for (int s = 0; s < nsys; ++s) {
        GB_REQUIRE(A[s] && d_B[s] && d_X[s], "pcg_solve_batched: system %d has a NULL pointer", s);
        GB_REQUIRE(k[s] >= 1 && k[s] <= KMAX, "pcg_solve_batched: k[%d]=%d not in 1..%d", s, k[s], KMAX);
    }
    PcgOptions o{};
    if (opt) o = *opt;
    if (!(o.tol > 0)) o.tol = 1e-10;
    int64_t nmax = 0;
    for (int s = 0; s < nsys; ++s) nmax = std::max<int64_t>(nmax, A[s]->n);
    if (o.max_iter <= 0) o.max_iter = 20 * nmax + 100;
    if (o.max_outer <= 0) o.max_outer = 30;
    if (!(o.inner_tol > 0)) o.inner_tol = 1e-4;
    if (o.check_every <= 0) o.check_every = 16;
    if (graphs_disabled()) o.use_graph = 0;
    GB_REQUIRE(o.precision >= GB_F64 && o.precision <= GB_F32_RU && o.precision != GB_BF16_RU,
               "pcg_solve_batched: precision must be GB_F64, GB_F32_IR, GB_BF16_IR or GB_F32_RU");
    GB_REQUIRE(o.precond == GB_PC_JACOBI, "pcg_solve_batched: the Jacobi preconditioner only");
    GB_REQUIRE(o.method == GB_CG, "pcg_solve_batched: CG only");
    for (int s = 0; s < nsys; ++s) {
        GB_REQUIRE((o.precision != GB_F32_IR && o.precision != GB_F32_RU) || A[s]->val32,
                   "pcg_solve_batched: system %d has no fp32 values", s);
        GB_REQUIRE(o.precision != GB_BF16_IR || A[s]->val16, "pcg_solve_batched: system %d has no bf16 values", s);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool ir = o.precision != GB_F64;
    Batch b;
    GB_TRY(setup_batch(b, nsys, A, d_B, d_X, k, o, st));

    cudaEvent_t e0, e1;
    GB_CHECK_CUDA(cudaEventCreate(&e0));
    GB_CHECK_CUDA(cudaEventCreate(&e1));
    GB_CHECK_CUDA(cudaEventRecord(e0, st));
    // R = B - A X0, ||B_j||, thresholds
    ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 1, o.x0_zero ? 1 : 0, o.tol);
    GB_CHECK_CUDA(cudaGetLastError());
    HostCols hc;
    GB_TRY(pull_cols(b, hc, st));
    std::vector<int> mask(nsys * KMAX, 0);
    std::vector<int> outer_cnt(nsys, 0);
    std::vector<long long> inner_its(nsys, 0);
    std::vector<long long> restarts(nsys, 0);
    std::vector<long long> fallback_its(nsys, 0);
    // small systems: solved whole by the persistent CTA-local kernel, one
    // launch for all of them; medium ones by the cluster kernel, one launch
    // for all of them; the loops below then find them converged (or take
    // over the columns they left above tol)
    std::vector<int> plist, clist, glist;
    for (int s = 0; s < nsys; ++s) {
        const int tier = o.persist_off == 1 ? 0 : persist_tier(A[s]->n, k[s]);
        if (tier == 1) plist.push_back(s);
        else if (tier == 2 && o.persist_off != 2) clist.push_back(s);
        else if (tier == 3 && o.persist_off == 3) glist.push_back(s);
    }
    if (!glist.empty()) {
        // one cooperative launch per group size (a system's group size depends
        // on its own size only, so its result does not depend on the batch)
        const int res = ir ? grid_resident_blocks<float>() : grid_resident_blocks<double>();
        std::map<int, std::vector<int>> by_g;
        for (int s : glist) by_g[grid_blocks_for(A[s]->n, kw_of(k[s]), std::max(res, 1))].push_back(s);
        for (auto &kv : by_g) {
            const int grc = res > 0 ? run_persist(b, kv.second, o, ir, st, 3) : 1;
            if (grc == 1) { glist.clear(); break; }  // not resident on this device: the loop takes them
            GB_TRY(grc);
        }
    }
    if (!clist.empty()) GB_TRY(run_persist(b, clist, o, ir, st, 2));
    for (int s : clist) plist.push_back(s);
    const size_t nsmall = plist.size() - clist.size();
    for (int s : glist) plist.push_back(s);
    if (!plist.empty()) {
        if (nsmall > 0) {
            std::vector<int> small(plist.begin(), plist.begin() + nsmall);
            GB_TRY(run_persist(b, small, o, ir, st, 1));
        }
        GB_TRY(pull_cols(b, hc, st));
        for (int *ep : b.grid_err) {
            int herr = 0;
            GB_CHECK_CUDA(cudaMemcpyAsync(&herr, ep, sizeof(int), cudaMemcpyDeviceToHost, st));
            GB_CHECK_CUDA(cudaStreamSynchronize(st));
            if (herr) {
                set_error("pcg_solve_batched: a grid-tier group barrier wait ran out");
                return GB_TIMEOUT;
            }
        }
        std::vector<BSys> hs(nsys);
        GB_CHECK_CUDA(cudaMemcpyAsync(hs.data(), b.d_sys, sizeof(BSys) * nsys, cudaMemcpyDeviceToHost, st));
        GB_CHECK_CUDA(cudaStreamSynchronize(st));
        for (int s : plist) {
            long long mx = 0;
            for (int j = 0; j < k[s]; ++j) mx = std::max(mx, hc.it[s][j]);
            if (ir) { inner_its[s] = mx; outer_cnt[s] = hs[s].outer; }
        }
    }
    int rc = GB_OK;
    if (!ir) {
        // fp64 recurrences; restart columns whose true residual misses tol
        for (int round = 0; round < 50; ++round) {
            bool any = false;
            for (int s = 0; s < nsys; ++s)
                for (int j = 0; j < k[s]; ++j) {
                    const bool need = hc.bb[s][j] > 0 && hc.rr[s][j] > o.tol * o.tol * hc.bb[s][j] &&
                                      (round == 0 || hc.status[s][j] == ST_CONV);
                    mask[s * KMAX + j] = need ? 1 : 0;
                    any |= need;
                    if (need && round > 0) restarts[s] += 1;
                }
            if (!any) break;
            rc = start_and_loop<double, double>(b, mask, o.max_iter, o, st);
            if (rc != GB_OK) break;
            ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 0, 0, o.tol);
            GB_CHECK_CUDA(cudaGetLastError());
            HostCols h2;
            rc = pull_cols(b, h2, st);
            if (rc != GB_OK) break;
            // keep status from the loop, residuals from the true residual
            for (int s = 0; s < nsys; ++s) { hc.rr[s] = h2.rr[s]; hc.status[s] = h2.status[s]; hc.it[s] = h2.it[s]; }
        }
    } else {
        rc = o.precision == GB_F32_RU   ? batched_ru<float>(b, o, st, outer_cnt, inner_its)
             : o.precision == GB_F32_IR ? batched_ir<float>(b, o, st, outer_cnt, inner_its)
                                        : batched_ir<__nv_bfloat16>(b, o, st, outer_cnt, inner_its);
        if (rc == GB_OK) rc = pull_cols(b, hc, st);
        // columns the refinement left above tol finish in fp64 from their X
        bool fb = false;
        for (int s2 = 0; s2 < nsys && rc == GB_OK; ++s2)
            for (int j = 0; j < k[s2]; ++j) {
                const bool need = hc.bb[s2][j] > 0 && hc.rr[s2][j] > o.tol * o.tol * hc.bb[s2][j];
                mask[s2 * KMAX + j] = need ? 1 : 0;
                fb |= need;
            }
        if (rc == GB_OK && fb) {
            for (int s2 = 0; s2 < nsys && rc == GB_OK; ++s2) {
                BSys &S = b.h[s2];
                const size_t nk = (size_t)S.A.n * S.k;
                double *P, *Q;
                rc = b.take(&P, nk);
                if (rc == GB_OK) rc = b.take(&Q, nk);
                if (rc != GB_OK) break;
                S.X = S.X64; S.R = S.R64; S.P = P; S.Q = Q; S.val = A[s2]->val;
                std::vector<long long> z(S.k, 0);
                cudaMemcpyAsync(S.c.it, z.data(), sizeof(long long) * S.k, cudaMemcpyHostToDevice, st);
                cudaStreamSynchronize(st);
            }
            if (rc == GB_OK) {
                cudaMemcpyAsync(b.d_sys, b.h.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, st);
                rc = start_and_loop<double, double>(b, mask, o.max_iter, o, st);
            }
            if (rc == GB_OK) {
                ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 0, 0, o.tol);
                HostCols h3;
                rc = pull_cols(b, h3, st);
                for (int s2 = 0; s2 < nsys && rc == GB_OK; ++s2) {
                    hc.rr[s2] = h3.rr[s2];
                    hc.status[s2] = h3.status[s2];
                    long long mx = 0;
                    for (int j = 0; j < k[s2]; ++j) if (mask[s2 * KMAX + j]) mx = std::max(mx, h3.it[s2][j]);
                    fallback_its[s2] = mx;
                }
            }
        }
    }
    if (rc != GB_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
    for (int s = 0; s < nsys; ++s) {
        const int g = stride_grid((int64_t)A[s]->n * k[s], 256, 8);
        ::gb::count_launches(1); k_scatter_rows<<<g, 256, 0, st>>>(A[s]->n, k[s], A[s]->perm, b.h[s].X64, d_X[s]);
    }
    GB_CHECK_CUDA(cudaEventRecord(e1, st));
    GB_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int worst = GB_OK;
    for (int s = 0; s < nsys; ++s) {
        PcgStats &S = stats[s];
        S = PcgStats{};
        double rel = 0.0, bn = 0.0;
        long long its = 0;
        int status = GB_OK;
        for (int j = 0; j < k[s]; ++j) {
            const double bb = hc.bb[s][j];
            const double r = bb > 0 ? std::sqrt(hc.rr[s][j] / bb) : 0.0;
            rel = std::max(rel, r);
            bn = std::max(bn, std::sqrt(bb));
            its = std::max(its, hc.it[s][j]);
            if (r > o.tol) status = (hc.status[s][j] == ST_BREAK) ? GB_BREAKDOWN : GB_NOT_CONVERGED;
        }
        S.iterations = ir ? inner_its[s] : its;
        S.restarts = restarts[s];
        S.outer = outer_cnt[s];
        S.relres = rel;
        S.bnorm = bn;
        S.status = status;
        S.solve_ms = ms;
        const double sv = ir ? (o.precision == GB_BF16_IR ? 2.0 : 4.0) : 8.0;
        const double sx = ir ? 4.0 : 8.0;
        S.bytes_moved = (double)S.iterations * ((double)A[s]->nnz * (sv + 4.0) + 7.0 * A[s]->n * k[s] * sx);
        S.kernel_launches = 3 * (S.iterations + fallback_its[s]);
        S.fallback_iterations = fallback_its[s];
        if (fallback_its[s]) S.bytes_moved += (double)fallback_its[s] * ((double)A[s]->nnz * 12.0 + 7.0 * A[s]->n * k[s] * 8.0);
        if (status != GB_OK && worst == GB_OK) worst = status;
    }
    if (worst != GB_OK) {
        set_error("pcg_solve_batched: a column did not reach tol (status %d)", worst);
        return worst;
    }
    return GB_OK;
}

// ------------------------------------------------------------ measurement --
// out (n x w, row-major) = columns j0 .. j0+w-1 of B (n x k, row-major)
__global__ void k_col_slice(int64_t n, int k, int j0, int w, const double *__restrict__ B, double *__restrict__ out) {
    const int64_t m = n * w;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / w;
        out[t] = B[r * k + j0 + (t - r * w)];
    }
}

extern "C" int pcg_batched_kernel_times(int nsys, const gb_sell *const *A, const double *const *d_B, const int *k,
                                        int precision, int iters, void *stream, double *h_ms) {
    GB_REQUIRE(nsys >= 1 && A && d_B && k && h_ms, "pcg_batched_kernel_times: NULL argument");
    GB_REQUIRE(iters >= 1 && iters <= 100000, "pcg_batched_kernel_times: iters must be in 1..100000");
    GB_REQUIRE(precision >= GB_F64 && precision <= GB_BF16_IR, "pcg_batched_kernel_times: bad precision");
    for (int s = 0; s < nsys; ++s) {
        GB_REQUIRE(A[s] && d_B[s], "pcg_batched_kernel_times: system %d has a NULL pointer", s);
        GB_REQUIRE(k[s] >= 1 && k[s] <= KMAX, "pcg_batched_kernel_times: k[%d]=%d not in 1..%d", s, k[s], KMAX);
        GB_REQUIRE(precision != GB_F32_IR || A[s]->val32, "pcg_batched_kernel_times: system %d has no fp32 values", s);
        GB_REQUIRE(precision != GB_BF16_IR || A[s]->val16, "pcg_batched_kernel_times: system %d has no bf16 values", s);
    }
    PcgOptions o{};
    o.precision = precision;
    o.x0_zero = 1;
    o.tol = 1e-10;
    cudaStream_t st = (cudaStream_t)stream;
    Batch b;
    GB_TRY(setup_batch(b, nsys, A, d_B, nullptr, k, o, st));
    // R = B, then the recurrences start on every column; thresholds below zero
    // keep every column iterating for the whole run
    ::gb::count_launches(1); k_bresid<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, 1, 1, o.tol);
    std::vector<int> mask((size_t)nsys * KMAX, 0);
    for (int s = 0; s < nsys; ++s)
        for (int j = 0; j < k[s]; ++j) mask[(size_t)s * KMAX + j] = 1;
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_mask, mask.data(), sizeof(int) * mask.size(), cudaMemcpyHostToDevice, st));
    HostCols hc;
    GB_TRY(pull_cols(b, hc, st));
    for (int s = 0; s < nsys; ++s) {
        std::vector<double> th(k[s], -1.0), sc(k[s]);
        for (int j = 0; j < k[s]; ++j) sc[j] = hc.rr[s][j] > 0 ? std::sqrt(hc.rr[s][j]) : 1.0;
        GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.thresh, th.data(), sizeof(double) * k[s], cudaMemcpyHostToDevice, st));
        GB_CHECK_CUDA(cudaMemcpyAsync(b.h[s].c.scale, sc.data(), sizeof(double) * k[s], cudaMemcpyHostToDevice, st));
    }
    if (precision == GB_F64) {
        ::gb::count_launches(1); k_bstart<double><<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, b.d_mask);
    } else {
        ::gb::count_launches(1); k_bscale_down<<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_mask);
        ::gb::count_launches(1); k_bstart<float><<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.partials, b.d_mask);
    }
    BGlobal g{};
    g.maxit = (long long)iters + 1;
    g.active_systems = nsys;
    g.budget = -1;
    GB_CHECK_CUDA(cudaMemcpyAsync(b.d_G, &g, sizeof(g), cudaMemcpyHostToDevice, st));
    GB_CHECK_CUDA(cudaGetLastError());
    std::vector<cudaEvent_t> ev(3 * (size_t)iters + 1);
    for (auto &e : ev) GB_CHECK_CUDA(cudaEventCreate(&e));
    cudaEventRecord(ev[0], st);
    for (int i = 0; i < iters; ++i) {
        for (int q = 0; q < 3; ++q) {
            if (precision == GB_F64) {
                if (q == 0) launch_bspmm<double, double>(b.tma, b.cls, b.units, b.d_sys, b.d_unit_sys, b.d_G, b.partials, st);
                else if (q == 1) { ::gb::count_launches(1); k_bupdate<double><<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_G, b.partials); }
                else { ::gb::count_launches(1); k_bpupdate<double><<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_G); }
            } else {
                if (q == 0) {
                    if (precision == GB_F32_IR) launch_bspmm<float, float>(b.tma, b.cls, b.units, b.d_sys, b.d_unit_sys, b.d_G, b.partials, st);
                    else launch_bspmm<float, __nv_bfloat16>(b.tma, b.cls, b.units, b.d_sys, b.d_unit_sys, b.d_G, b.partials, st);
                } else if (q == 1) { ::gb::count_launches(1); k_bupdate<float><<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_G, b.partials); }
                else { ::gb::count_launches(1); k_bpupdate<float><<<b.units, NT, 0, st>>>(b.d_sys, b.d_unit_sys, b.d_G); }
            }
            cudaEventRecord(ev[3 * (size_t)i + q + 1], st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev.back());
    double tot[3] = {0, 0, 0};
    for (int i = 0; i < iters && e == cudaSuccess; ++i)
        for (int q = 0; q < 3; ++q) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[3 * (size_t)i + q], ev[3 * (size_t)i + q + 1]);
            tot[q] += ms;
        }
    for (auto &x : ev) cudaEventDestroy(x);
    if (e != cudaSuccess) { set_error("pcg_batched_kernel_times: %s", cudaGetErrorString(e)); return GB_ECUDA; }
    BGlobal hg{};
    GB_CHECK_CUDA(cudaMemcpyAsync(&hg, b.d_G, sizeof(hg), cudaMemcpyDeviceToHost, st));
    GB_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < 3; ++q) h_ms[q] = tot[q] / iters;
    if (hg.done) {
        set_error("pcg_batched_kernel_times: the recurrences stopped early; use fewer iterations");
        return GB_BREAKDOWN;
    }
    return GB_OK;
}

// RHS block width autotuner: for each width w in {1, 2, 4, 8, 16, 32} (w <= k)
// the k columns are cut into ceil(k/w) systems of at most w columns (the last
// one shorter), one blocked iteration of that batch is timed with
// pcg_batched_kernel_times (2 warm-up + 8 timed iterations), and the width
// with the least time per column wins.
extern "C" int pcg_batched_autotune_width(const gb_sell *A, const double *d_B, int k, int precision, void *stream,
                                          int *best_width, double *h_ms) {
    GB_REQUIRE(A && d_B && best_width, "pcg_batched_autotune_width: NULL argument");
    GB_REQUIRE(k >= 1 && k <= 256, "pcg_batched_autotune_width: k=%d not in 1..256", k);
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = A->n;
    Mem mem(nullptr, st);
    double *tmp = nullptr;
    GB_TRY(mem.alloc_n(&tmp, (size_t)n * k));
    struct Guard { Mem &m; double *p; ~Guard() { m.release(p); } } guard{mem, tmp};
    double best = 1e300;
    *best_width = 0;
    const int widths[6] = {1, 2, 4, 8, 16, 32};
    for (int wi = 0; wi < 6; ++wi) {
        const int w = widths[wi];
        if (w > k) break;
        std::vector<const gb_sell *> As;
        std::vector<const double *> Bs;
        std::vector<int> ks;
        for (int j0 = 0; j0 < k; j0 += w) {
            const int ww = std::min(w, k - j0);
            double *dst = tmp + (size_t)n * j0;
            ::gb::count_launches(1);
            k_col_slice<<<stride_grid(n * ww, 256, 8), 256, 0, st>>>(n, k, j0, ww, d_B, dst);
            As.push_back(A);
            Bs.push_back(dst);
            ks.push_back(ww);
        }
        GB_CHECK_CUDA(cudaGetLastError());
        double ms[3] = {0, 0, 0};
        GB_TRY(pcg_batched_kernel_times((int)As.size(), As.data(), Bs.data(), ks.data(), precision, 2, stream, ms));
        GB_TRY(pcg_batched_kernel_times((int)As.size(), As.data(), Bs.data(), ks.data(), precision, 8, stream, ms));
        const double t = ms[0] + ms[1] + ms[2];
        if (h_ms) h_ms[wi] = t;
        if (t < best) { best = t; *best_width = w; }
    }
    for (int wi = 0; wi < 6 && h_ms; ++wi)
        if (widths[wi] > k) h_ms[wi] = 0.0;
    return GB_OK;
}

// ------------------------------------------------------------- grid tier --
// One fp64 system (one right-hand side) solved whole by one persistent
// launch: one thread-block cluster (n <= 2^16, hardware cluster barriers) or
// one group of the grid tier (a cooperative launch).  A single workspace
// allocation (stream-ordered), the permuted b and x0 gathered, the launch --
// which forms r = b - A x0, ||b|| and the threshold itself and runs the CG
// rounds with true-residual restarts --, x scattered back, and one copy of
// the column state to the host.  Returns 1 (nothing done) when the grid
// kernel cannot be resident on this device.
int gb::grid_solve_single(const gb_sell *M, const double *d_b, double *d_x, const PcgOptions &o, cudaStream_t st,
                          PcgStats *stats) {
    const int64_t n = M->n;
    const bool cluster = n <= GB_CLUSTER_SINGLE_MAX && o.persist_off != 3;
    const int res = cluster ? CLUSTER_CS : grid_resident_blocks<double>();
    if (res <= 0) return 1;
    const int G = cluster ? CLUSTER_CS : grid_blocks_for(n, 1, res);
    // workspace: [BSys | cd | ci | cs | list, next | grid ws | B64 X64 R64 P Q]
    const size_t o_sys = 0;
    const size_t o_cd = o_sys + align256(sizeof(BSys));
    const size_t o_ci = o_cd + align256(sizeof(double) * 10 * KMAX);
    const size_t o_cs = o_ci + align256(sizeof(long long) * KMAX);
    const size_t o_lst = o_cs + align256(sizeof(int) * 2 * KMAX);
    const size_t o_ws = o_lst + 256;
    const size_t o_vec = o_ws + grid_ws_bytes(1, G);
    const size_t bytes = o_vec + 5 * align256(sizeof(double) * (size_t)n);
    char *ws = nullptr;
    {
        const cudaError_t e = cudaMallocAsync((void **)&ws, bytes, st);
        if (e != cudaSuccess) {
            set_error("pcg_solve (grid tier): cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? GB_ENOMEM : GB_ECUDA;
        }
        count_device_alloc();
    }
    struct Free {
        char *p;
        cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{ws, st};
    const size_t vb = align256(sizeof(double) * (size_t)n);
    double *B64 = (double *)(ws + o_vec), *X64 = (double *)(ws + o_vec + vb), *R64 = (double *)(ws + o_vec + 2 * vb);
    double *P = (double *)(ws + o_vec + 3 * vb), *Q = (double *)(ws + o_vec + 4 * vb);
    BSys h{};
    h.A = M->view();
    h.val = M->val;
    h.X = X64; h.R = R64; h.P = P; h.Q = Q;
    h.B64 = B64; h.X64 = X64; h.R64 = R64;
    double *cd = (double *)(ws + o_cd);
    h.c.rho = cd; h.c.pq = cd + KMAX; h.c.alpha = cd + 2 * KMAX; h.c.beta = cd + 3 * KMAX;
    h.c.rr = cd + 4 * KMAX; h.c.bb = cd + 5 * KMAX; h.c.thresh = cd + 6 * KMAX; h.c.scale = cd + 7 * KMAX;
    h.c.pz = cd + 8 * KMAX; h.c.target = cd + 9 * KMAX;
    h.c.it = (long long *)(ws + o_ci);
    h.c.done = (int *)(ws + o_cs);
    h.c.status = (int *)(ws + o_cs) + KMAX;
    h.k = 1;
    h.kw = 1;
    h.unit0 = 0;
    h.nunits = 1;
    h.rows_per_unit = n;
    h.active = 1;
    GB_CHECK_CUDA(cudaMemsetAsync(ws, 0, o_vec, st));
    GB_CHECK_CUDA(cudaMemcpyAsync(ws + o_sys, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GB_CHECK_CUDA(cudaEventCreate(&e0));
    GB_CHECK_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evs{e0, e1};
    GB_CHECK_CUDA(cudaEventRecord(e0, st));
    const int g = stride_grid(n, 256, 8);
    ::gb::count_launches(1); k_gather_rows<<<g, 256, 0, st>>>(n, 1, M->perm, d_b, B64);
    ::gb::count_launches(1); k_gather_rows<<<g, 256, 0, st>>>(n, 1, M->perm, o.x0_zero ? nullptr : d_x, X64);
    GB_CHECK_CUDA(cudaGetLastError());
    PersistOpts po{};
    po.tol = o.tol;
    po.maxit = o.max_iter;
    po.max_outer = 50;
    po.init = 1;
    po.x0_zero = o.x0_zero ? 1 : 0;
    int *list = (int *)(ws + o_lst), *next = list + 1;
    int *d_err = nullptr;
    if (cluster) {
        // the grid workspace's error word stays zero: a cluster's barriers are hardware ones
        d_err = grid_ws_err(ws + o_ws, 1, G);
        ::gb::count_launches(1);
        k_bcluster<double><<<CLUSTER_CS, PNT, 0, st>>>((BSys *)(ws + o_sys), list, 1, next, po);
        GB_CHECK_CUDA(cudaGetLastError());
    } else {
        GB_TRY(launch_grid<double>((BSys *)(ws + o_sys), list, 1, next, G, 1, ws + o_ws, po, st, &d_err));
    }
    ::gb::count_launches(1); k_scatter_rows<<<g, 256, 0, st>>>(n, 1, M->perm, X64, d_x);
    GB_CHECK_CUDA(cudaGetLastError());
    GB_CHECK_CUDA(cudaEventRecord(e1, st));
    // column state, the tier's round count and the error word
    std::vector<char> hb(o_ws);
    int herr = 0;
    GB_CHECK_CUDA(cudaMemcpyAsync(hb.data(), ws, o_ws, cudaMemcpyDeviceToHost, st));
    GB_CHECK_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CHECK_CUDA(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const BSys *hs = (const BSys *)(hb.data() + o_sys);
    const double *hcd = (const double *)(hb.data() + o_cd);
    const long long it = ((const long long *)(hb.data() + o_ci))[0];
    const int done = ((const int *)(hb.data() + o_cs))[0];
    const int status = ((const int *)(hb.data() + o_cs))[KMAX];
    const double rr = hcd[4 * KMAX], bb = hcd[5 * KMAX];
    *stats = PcgStats{};
    stats->iterations = it;
    stats->restarts = hs->outer > 1 ? hs->outer - 1 : 0;
    stats->bnorm = std::sqrt(bb);
    stats->relres = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    stats->solve_ms = ms;
    stats->kernel_launches = 4;
    stats->bytes_moved = (double)it * ((double)M->nnz * 12.0 + 7.0 * (double)n * 8.0);
    if (herr || !done) stats->status = GB_TIMEOUT;
    else if (bb == 0.0 || stats->relres <= o.tol) stats->status = GB_OK;
    else if (status == ST_BREAK) stats->status = GB_BREAKDOWN;
    else if (status == ST_TIMEOUT) stats->status = GB_TIMEOUT;
    else stats->status = GB_NOT_CONVERGED;
    if (bb == 0.0) {  // b = 0: x = 0 (the kernel ran no round; X64 holds x0)
        GB_CHECK_CUDA(cudaMemsetAsync(d_x, 0, sizeof(double) * (size_t)n, st));
        stats->relres = 0.0;
    }
    return GB_OK;
}

// A group exchange that must run out: one block launched of a group of two,
// so the second block's exchange number never appears and the first one's
// wait ends on its time limit -- through the grid kernel itself, with an
// empty list (no system is touched).
extern "C" int gbpcg_grid_wait_selftest(double limit_ms, void *stream, double *h_waited_ms) {
    GB_REQUIRE(limit_ms > 0.0 && limit_ms <= 2000.0, "gbpcg_grid_wait_selftest: limit_ms must be in (0, 2000]");
    cudaStream_t st = (cudaStream_t)stream;
    const int G = 2;
    const size_t o_ws = 256;
    const size_t bytes = o_ws + grid_ws_bytes(1, G);
    char *ws = nullptr;
    GB_CHECK_CUDA(cudaMalloc((void **)&ws, bytes));
    count_device_alloc();
    int *list = (int *)ws, *next = list + 1;
    GB_CHECK_CUDA(cudaMemsetAsync(ws, 0, bytes, st));
    PersistOpts po{};
    po.wait_ns = (unsigned long long)(limit_ms * 1e6);
    double *gslots = (double *)(ws + o_ws);
    int *err = grid_ws_err(ws + o_ws, 1, G);
    BSys *no_sys = nullptr;
    int nlist = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    // one block launched of a group of two: the barrier's second arrival never comes
    ::gb::count_launches(1);
    k_bgrid<double><<<1, PNT, 0, st>>>(no_sys, list, nlist, next, gslots, G, err, po);
    cudaError_t e = cudaGetLastError();
    cudaEventRecord(e1, st);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ws);
    if (e != cudaSuccess) { set_error("gbpcg_grid_wait_selftest: %s", cudaGetErrorString(e)); return GB_ECUDA; }
    if (h_waited_ms) *h_waited_ms = ms;
    if (herr) {
        set_error("gbpcg_grid_wait_selftest: the group barrier gave up after %.3f ms", (double)ms);
        return GB_TIMEOUT;
    }
    return GB_OK;
}
