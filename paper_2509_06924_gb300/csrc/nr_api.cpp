// nr_api.cpp -- host side of the C ABI declared in include/nr.h: argument
// and metadata validation, the library's own Gauss-Hermite rule, plans (the
// per-batch device work lists, cached by metadata), launch-shape choice and
// autotuning, host-memory staging, and the device status word.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "nr.h"
#include "nr_internal.h"

using namespace nrimpl;

namespace {

thread_local std::string g_last_error;

nr_status fail(nr_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define NR_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(e_ == cudaErrorMemoryAllocation ? NR_ENOMEM : NR_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                      \
    } while (0)

// ------------------------------------------------------------ quadrature --
// Gauss-Hermite rule for exp(-x^2) by Golub-Welsch: the nodes are the
// eigenvalues of the symmetric tridiagonal Jacobi matrix of the Hermite
// recurrence (off-diagonal sqrt(j/2)), found here by cyclic Jacobi rotations;
// each node is then polished by Newton steps on the orthonormal recurrence
// and its weight taken as 2 / psi_K'(x)^2.
double herm_psi(int K, double x, double *dpsi)
{
    double pm1 = 0.0, p = 1.0 / std::sqrt(std::sqrt(M_PI));
    for (int j = 0; j < K; ++j) {
        const double pn = x * std::sqrt(2.0 / (j + 1)) * p - std::sqrt((double)j / (j + 1)) * pm1;
        pm1 = p;
        p = pn;
    }
    *dpsi = std::sqrt(2.0 * K) * pm1;
    return p;
}

bool gauss_hermite(int K, double *x, double *w)
{
    if (K < 1 || K > NR_MAX_QUAD) return false;
    // fixed-size storage: no heap allocation (nr_loglik_grad_noalloc uses this)
    double A[NR_MAX_QUAD * NR_MAX_QUAD] = {};
    for (int i = 0; i + 1 < K; ++i) A[i * K + i + 1] = A[(i + 1) * K + i] = std::sqrt((i + 1) / 2.0);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) off += A[p * K + q] * A[p * K + q];
        if (off < 1e-30) break;
        for (int p = 0; p < K; ++p)
            for (int q = p + 1; q < K; ++q) {
                const double apq = A[p * K + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[q * K + q] - A[p * K + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < K; ++k) { // columns p, q
                    const double akp = A[k * K + p], akq = A[k * K + q];
                    A[k * K + p] = c * akp - s * akq;
                    A[k * K + q] = s * akp + c * akq;
                }
                for (int k = 0; k < K; ++k) { // rows p, q
                    const double apk = A[p * K + k], aqk = A[q * K + k];
                    A[p * K + k] = c * apk - s * aqk;
                    A[q * K + k] = s * apk + c * aqk;
                }
            }
    }
    double nodes[NR_MAX_QUAD];
    for (int i = 0; i < K; ++i) nodes[i] = A[i * K + i];
    std::sort(nodes, nodes + K);
    for (int i = 0; i < K; ++i) {
        double xi = nodes[i], d;
        for (int it = 0; it < 3; ++it) {
            const double f = herm_psi(K, xi, &d);
            if (d != 0.0) xi -= f / d;
        }
        herm_psi(K, xi, &d);
        x[i] = xi;
        w[i] = 2.0 / (d * d);
    }
    return true;
}

// --------------------------------------------------------------- buffers --
// Allocation-failure injection for tests (nr_debug_fail_allocs): the next
// g_fail_allocs device allocations of the library report
// cudaErrorMemoryAllocation without calling cudaMalloc.
std::atomic<int> g_fail_allocs{0};

cudaError_t dev_malloc(void **p, size_t n)
{
    int k = g_fail_allocs.load();
    while (k > 0 && !g_fail_allocs.compare_exchange_weak(k, k - 1)) {
    }
    if (k > 0) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, n);
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t ensure(size_t n)
    {
        if (n <= bytes) return cudaSuccess;
        if (p) {
            cudaDeviceSynchronize();
            cudaFree(p);
            p = nullptr;
            bytes = 0;
        }
        cudaError_t e = dev_malloc(&p, n);
        if (e == cudaSuccess) bytes = n;
        else p = nullptr;
        return e;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// NVTX range around a library call (no cost without a profiler attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

constexpr int kGradBuckets[] = {1, 2, 4, 8, 12, 16, 20, 32, 64};

// Register buckets: the 1-layer kernels are specialised for exactly one
// layer (the common thin-film case); bare substrates go to the 2 bucket.
int grad_bucket(int n)
{
    if (n == 1) return 1;
    for (int b : kGradBuckets)
        if (b > 1 && n <= b) return b;
    return -1;
}
// Forward (model, log-likelihood) buckets: exactly one layer; up to 20 layers
// (the paired runtime-n kernel, whose log-likelihood mode takes the
// special-function unit's sin / cos); deeper stacks (64: the one-evaluation
// runtime-n kernel, table sin / cos in every mode, since the special-function
// unit's phase error accumulates over that many layers)
int fwd_bucket(int n) { return n == 1 ? 1 : n <= 20 ? 0 : 64; }

struct Group {
    int nmax = 0;
    int item_begin = 0;
    int item_count = 0;
    int grid = 0;
    int tile_q = 0;
    bool pair = true; // the paired kernel where it applies (the autotuner may clear it)
};

// Work list of one mode family (forward = model/loglik, or gradient).
struct WorkList {
    std::vector<Group> groups;
    DevBuf d_stacks, d_items, d_partials, d_done, d_ticket;
    int64_t partial_doubles = 0;
    int chunk_q = 0;
    bool tuned = false; // launch shapes chosen by timing (nr_plan, autotune = 1)
};

struct Plan {
    // key
    int32_t S = 0, D = 0, K = 0;
    std::vector<int32_t> n_layers, dataset;
    std::vector<int64_t> q_off;
    // derived
    int64_t total_params = 0, total_out = 0, total_q = 0, evals = 0;
    WorkList fwd, grad;
    bool fwd_built = false, grad_built = false;
    // FP64 plain path
    DevBuf d64_stacks, d64_items, d64_llpert;
    int n64_items = 0, n64_pert = 1;
    bool fp64_built = false;
    uint64_t last_use = 0;
};



} // namespace

namespace nrimpl {
// Message for nr_last_error() from the other translation units.
void record_error(const char *msg) { g_last_error = msg; }

bool make_quad_const(int K, QuadConst &qc)
{
    double x[NR_MAX_QUAD], w[NR_MAX_QUAD];
    if (!gauss_hermite(K, x, w)) return false;
    const double c = 1.0 / (2.0 * std::sqrt(std::log(2.0)));
    const double isp = 1.0 / std::sqrt(M_PI);
    qc = QuadConst{};
    qc.K = K;
    for (int k = 0; k < K; ++k) {
        const double g = x[k] * c;
        qc.gd[k] = g;
        qc.g_hi[k] = (float)g;
        qc.g_lo[k] = (float)(g - (double)(float)g);
        qc.wd[k] = w[k] * isp;
        qc.w[k] = (float)(w[k] * isp);
    }
    for (int i = 0; i < kSinCosTabN; ++i) {
        const double a = 2.0 * M_PI * i / kSinCosTabN;
        qc.cs_tab[i] = (float)std::cos(a);
        qc.cs_tab[kSinCosTabN + i] = (float)std::sin(a);
    }
    return true;
}
} // namespace nrimpl

struct nr_ctx {
    int device = 0;
    int sms = 0;
    char gpu_name[256] = {};
    nr_options opt{};
    QuadConst qc{};
    int32_t *d_status = nullptr;
    std::vector<std::unique_ptr<Plan>> plans;
    uint64_t clock = 0;
    // side streams and events of the concurrent register-bucket launches
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    // host-memory staging
    DevBuf s_params, s_q, s_dq, s_robs, s_rerr, s_out, s_ll, s_grad, s_res;
    DevBuf p_off, p_nl, p_z, p_rho, p_iota; // SLD-profile metadata and host-call staging
    WorkItem poisoned{-1, 0, 0, 0};         // nr_debug_poison_plan: the item it replaced
};

// On-device HMC sampler: the replicated likelihood batch of C chains x
// n_contrasts stacks and the per-chain workspaces (see nr_hmc.cu).
struct nr_sampler {
    nr_ctx *ctx = nullptr;
    int device = 0;
    int C = 0, P = 0, NC = 0, NS = 0;
    std::vector<int32_t> n_layers, dataset; // [C * NC], chain-major
    std::vector<int64_t> q_off;
    nr_batch batch{};
    DevBuf d_src, d_val, d_lo, d_hi, d_tie_ptr, d_tie_slot, d_params, d_ll, d_gpk, d_mom, d_u0, d_H0, d_lp0;
    DevBuf d_vu, d_vg, d_vlp, d_vpart; // variational step: u = mu + L e, d log pi / du, log pi, ELBO part
    DevBuf d_vbias;                    // Adam bias corrections of the current iteration (2 doubles)
    int res_param = -1;                // free parameter scaling every dQ (-1: none)
    DevBuf d_dqs, d_gres;              // per stack: that scale, d loglik / d ln(scale)
};

namespace {

nr_status validate(const nr_batch *b)
{
    if (!b) return fail(NR_EINVAL, "batch is NULL");
    if (b->n_stacks < 0) return fail(NR_EINVAL, "n_stacks < 0");
    if (b->memory != NR_MEM_DEVICE && b->memory != NR_MEM_HOST) return fail(NR_EINVAL, "bad memory kind");
    if (b->n_stacks == 0) return NR_OK;
    if (b->n_datasets < 1) return fail(NR_EINVAL, "n_datasets < 1");
    if (!b->n_layers || !b->dataset || !b->q_off) return fail(NR_EINVAL, "metadata pointer is NULL");
    if (!b->params || !b->q || !b->dq) return fail(NR_EINVAL, "params/q/dq pointer is NULL");
    if (b->q_off[0] != 0) return fail(NR_EINVAL, "q_off[0] != 0");
    for (int d = 0; d < b->n_datasets; ++d) {
        const int64_t len = b->q_off[d + 1] - b->q_off[d];
        if (len < 0) return fail(NR_EINVAL, "q_off not non-decreasing at dataset %d", d);
        if (len > (int64_t)1 << 30) return fail(NR_EINVAL, "dataset %d too long", d);
    }
    for (int s = 0; s < b->n_stacks; ++s) {
        if (b->n_layers[s] < 0 || b->n_layers[s] > NR_MAX_LAYERS)
            return fail(NR_EINVAL, "stack %d: n_layers %d outside [0, %d]", s, b->n_layers[s], NR_MAX_LAYERS);
        if (b->dataset[s] < 0 || b->dataset[s] >= b->n_datasets)
            return fail(NR_EINVAL, "stack %d: dataset %d outside [0, %d)", s, b->dataset[s], b->n_datasets);
    }
    return NR_OK;
}

bool same_meta(const Plan &p, const nr_batch *b, int K)
{
    if (p.S != b->n_stacks || p.D != b->n_datasets || p.K != K) return false;
    if (p.S == 0) return true;
    return std::memcmp(p.n_layers.data(), b->n_layers, sizeof(int32_t) * p.S) == 0 &&
           std::memcmp(p.dataset.data(), b->dataset, sizeof(int32_t) * p.S) == 0 &&
           std::memcmp(p.q_off.data(), b->q_off, sizeof(int64_t) * (p.D + 1)) == 0;
}

// Cutting stacks into Q-range chunks.  The register buckets of a work list
// run concurrently, so their chunk lengths are chosen together: for a bound
// B on the cost of any one item, every bucket takes its longest chunk (a
// multiple of its tile, or the whole dataset) whose items stay within B, and
// the estimated makespan is Graham's bound for longest-first queues, the
// summed cost of all items / resident CTAs + B.  An item costs (n + 1) x its
// Q points x K layer-evaluations plus a fixed overhead (queue ticket,
// staging, reductions, output) of about kItemOverhead layer-evaluations
// (measured: about 4 us of a CTA's time on the one-layer kernels), twice
// that for a chunk of a cut stack (partial sums, arrival counter, the last
// arriver's sum).  The best B must beat whole stacks by 10 %; batches with
// kChunkWaves stacks per resident CTA keep whole stacks without the search.
constexpr int64_t kChunkWaves = 8;
constexpr double kItemOverhead = 1000.0;

struct GroupSpan {
    int nmax;
    size_t i0, i1;  // range of `order`
    int tile_q;
    int64_t resident;
};

// One chunk length of a group with its summed item cost, largest item cost
// and item count
struct ChunkCand {
    int64_t chunk;
    double total, big;
};

std::vector<int64_t> choose_chunks(const Plan &pl, const std::vector<int> &order, const std::vector<GroupSpan> &gs)
{
    std::vector<int64_t> whole(gs.size(), 1);
    int64_t nst = 0;
    double res_w = 0.0, w_sum = 0.0;
    std::vector<std::vector<ChunkCand>> cands(gs.size());
    const double O = kItemOverhead / std::max(pl.K, 1); // in (n + 1) x Q units
    auto dlen = [&](int s) { return pl.q_off[pl.dataset[s] + 1] - pl.q_off[pl.dataset[s]]; };
    auto cost_of = [&](const GroupSpan &g, int64_t chunk) {
        ChunkCand c{chunk, 0.0, 0.0};
        for (size_t i = g.i0; i < g.i1; ++i) {
            const int s = order[i];
            const int64_t len = dlen(s);
            const int64_t nch = std::max<int64_t>(1, (len + chunk - 1) / chunk);
            const double o = nch > 1 ? 2.0 * O : O, w = pl.n_layers[s] + 1.0;
            c.total += w * (double)len + (double)nch * o;
            c.big = std::max(c.big, w * (double)std::min(chunk, std::max<int64_t>(len, 1)) + o);
        }
        return c;
    };
    for (size_t k = 0; k < gs.size(); ++k) {
        int64_t max_len = 1;
        for (size_t i = gs[k].i0; i < gs[k].i1; ++i) max_len = std::max(max_len, dlen(order[i]));
        whole[k] = max_len;
        nst += (int64_t)(gs[k].i1 - gs[k].i0);
        const ChunkCand w = cost_of(gs[k], max_len);
        res_w += w.total * (double)gs[k].resident;
        w_sum += w.total;
        cands[k].push_back(w);
    }
    // resident CTAs of the concurrent launches: their cost-weighted mean
    const double R = w_sum > 0.0 ? std::max(1.0, res_w / w_sum) : 1.0;
    if ((double)nst >= (double)kChunkWaves * R) return whole;
    for (size_t k = 0; k < gs.size(); ++k)
        // chunk lengths of 1..16 tiles, then growing by a quarter (a few
        // dozen candidates however long the datasets are)
        for (int64_t mt = 1; mt * gs[k].tile_q < whole[k]; mt = mt < 16 ? mt + 1 : mt + (mt + 3) / 4)
            cands[k].push_back(cost_of(gs[k], mt * gs[k].tile_q));
    // the makespan estimate for a bound B on the largest item
    auto est = [&](double B, std::vector<int64_t> *pick) {
        double total = 0.0, big = 0.0;
        for (size_t k = 0; k < gs.size(); ++k) {
            const ChunkCand *sel = nullptr;
            for (const ChunkCand &c : cands[k])
                if (c.big <= B && (!sel || c.chunk > sel->chunk)) sel = &c;
            if (!sel) return -1.0;
            total += sel->total;
            big = std::max(big, sel->big);
            if (pick) (*pick)[k] = sel->chunk;
        }
        return total / R + big;
    };
    double whole_est = 0.0;
    {
        double total = 0.0, big = 0.0;
        for (size_t k = 0; k < gs.size(); ++k) {
            total += cands[k][0].total;
            big = std::max(big, cands[k][0].big);
        }
        whole_est = total / R + big;
    }
    double best_est = whole_est, best_B = -1.0;
    for (size_t k = 0; k < gs.size(); ++k)
        for (const ChunkCand &c : cands[k]) {
            const double e = est(c.big, nullptr);
            if (e >= 0.0 && e < best_est) {
                best_est = e;
                best_B = c.big;
            }
        }
    if (best_B < 0.0 || best_est >= 0.9 * whole_est) return whole;
    std::vector<int64_t> pick(gs.size(), 1);
    est(best_B, &pick);
    return pick;
}

int tile_for(const nr_ctx *ctx, int mode, int nmax)
{
    int tq = mixed_tile_q(mode, nmax, ctx->qc.K);
    if (ctx->opt.tile_q > 0) tq = std::min(tq, ctx->opt.tile_q);
    return std::max(tq, 1);
}

// Side streams (non-blocking) and events for launching `groups` register
// buckets concurrently; created while a plan is built, i.e. before any
// stream capture of the calls that use them.
nr_status ensure_side_streams(nr_ctx *ctx, size_t groups)
{
    if (groups < 2 || ctx->opt.serial) return NR_OK;
    if (!ctx->ev_fork) NR_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    while (ctx->side.size() + 1 < groups) {
        cudaStream_t s = nullptr;
        NR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ctx->side.push_back(s);
    }
    while (ctx->ev_join.size() + 1 < groups) {
        cudaEvent_t e = nullptr;
        NR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->ev_join.push_back(e);
    }
    return NR_OK;
}

// Build the work list of one mode family: stacks grouped by register bucket,
// each stack cut into chunks when there are too few stacks to fill the GPU,
// items of a group ordered by decreasing cost (longest-processing-time first
// for the persistent queue).
nr_status build_worklist(nr_ctx *ctx, Plan &pl, int mode, WorkList &wl)
{
    const int S = pl.S;
    std::vector<int> bucket(S);
    for (int s = 0; s < S; ++s)
        bucket[s] = is_grad_mode(mode) ? grad_bucket(pl.n_layers[s]) : fwd_bucket(pl.n_layers[s]);
    std::vector<int> order(S);
    for (int s = 0; s < S; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bucket[a] < bucket[b]; });

    std::vector<StackInfo> info(S);
    std::vector<WorkItem> items;
    int64_t par = 0, out = 0;
    std::vector<int64_t> par_off(S), out_off(S);
    for (int s = 0; s < S; ++s) {
        par_off[s] = par;
        out_off[s] = out;
        par += 4 * (int64_t)pl.n_layers[s] + 6;
        out += pl.q_off[pl.dataset[s] + 1] - pl.q_off[pl.dataset[s]];
    }
    wl.groups.clear();
    // the register buckets (ranges of `order`) with their launch shapes
    std::vector<GroupSpan> spans;
    for (size_t i0 = 0; i0 < order.size();) {
        size_t i1 = i0;
        const int b = bucket[order[i0]];
        while (i1 < order.size() && bucket[order[i1]] == b) ++i1;
        int occ = 0;
        cudaError_t e = mixed_occupancy(mode, b, ctx->qc.K, &occ);
        if (e != cudaSuccess) return fail(NR_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
        spans.push_back(GroupSpan{b, i0, i1, tile_for(ctx, mode, b), (int64_t)ctx->sms * std::max(occ, 1)});
        i0 = i1;
    }
    std::vector<int64_t> chunks = ctx->opt.chunk_q > 0 ? std::vector<int64_t>(spans.size(), ctx->opt.chunk_q)
                                                       : choose_chunks(pl, order, spans);
    int64_t part = 0;
    wl.chunk_q = 0;
    for (size_t k = 0; k < spans.size(); ++k) {
        const GroupSpan &sp = spans[k];
        Group g;
        g.nmax = sp.nmax;
        g.tile_q = sp.tile_q;
        const int64_t chunk = std::max<int64_t>(chunks[k], 1);
        wl.chunk_q = std::max(wl.chunk_q, (int)std::min<int64_t>(chunk, 1 << 30));
        g.item_begin = (int)items.size();
        std::vector<std::pair<int64_t, WorkItem>> gi;
        for (size_t i = sp.i0; i < sp.i1; ++i) {
            const int s = order[i];
            const int nq = (int)(pl.q_off[pl.dataset[s] + 1] - pl.q_off[pl.dataset[s]]);
            const int nch = std::max(1, (int)((nq + chunk - 1) / chunk));
            StackInfo &si = info[s];
            si.par_off = par_off[s];
            si.out_off = out_off[s];
            si.q_begin = pl.q_off[pl.dataset[s]];
            si.n = pl.n_layers[s];
            si.nq = nq;
            si.n_chunks = nch;
            si.part_base = nch > 1 ? part : 0;
            si.pad = 0;
            if (nch > 1) part += (int64_t)nch * n_slot(si.n);
            for (int c = 0; c < nch; ++c) {
                WorkItem w;
                w.stack = s;
                w.q_lo = (int)std::min<int64_t>((int64_t)c * chunk, nq);
                w.q_hi = (int)std::min<int64_t>((int64_t)(c + 1) * chunk, nq);
                w.chunk = c;
                const int64_t cost = (int64_t)(si.n + 1) * (w.q_hi - w.q_lo) + 1;
                gi.push_back({cost, w});
            }
        }
        std::stable_sort(gi.begin(), gi.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
        for (auto &x : gi) items.push_back(x.second);
        g.item_count = (int)items.size() - g.item_begin;
        g.grid = (int)std::min<int64_t>(g.item_count, sp.resident);
        if (ctx->opt.grid_ctas > 0) g.grid = std::min(g.item_count, ctx->opt.grid_ctas);
        g.grid = std::max(g.grid, 1);
        wl.groups.push_back(g);
    }
    wl.partial_doubles = part;
    NR_CUDA(wl.d_stacks.ensure(sizeof(StackInfo) * std::max(S, 1)));
    NR_CUDA(wl.d_items.ensure(sizeof(WorkItem) * std::max<size_t>(items.size(), 1)));
    NR_CUDA(wl.d_partials.ensure(sizeof(double) * std::max<int64_t>(part, 1)));
    NR_CUDA(wl.d_done.ensure(sizeof(int32_t) * std::max(S, 1)));
    NR_CUDA(wl.d_ticket.ensure(sizeof(int32_t) * 2 * std::max<size_t>(wl.groups.size(), 1)));
    NR_CUDA(cudaMemcpy(wl.d_stacks.p, info.data(), sizeof(StackInfo) * S, cudaMemcpyHostToDevice));
    if (!items.empty())
        NR_CUDA(cudaMemcpy(wl.d_items.p, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice));
    NR_CUDA(cudaMemset(wl.d_done.p, 0, sizeof(int32_t) * std::max(S, 1)));
    NR_CUDA(cudaMemset(wl.d_ticket.p, 0, sizeof(int32_t) * 2 * std::max<size_t>(wl.groups.size(), 1)));
    return ensure_side_streams(ctx, wl.groups.size());
}

nr_status build_fp64(nr_ctx *ctx, Plan &pl)
{
    (void)ctx;
    const int S = pl.S;
    std::vector<StackInfo> info(S);
    std::vector<WorkItem> items;
    int64_t par = 0, out = 0, slot = 0;
    int maxp = 0;
    for (int s = 0; s < S; ++s) {
        StackInfo &si = info[s];
        const int nq = (int)(pl.q_off[pl.dataset[s] + 1] - pl.q_off[pl.dataset[s]]);
        si.par_off = par;
        si.out_off = out;
        si.q_begin = pl.q_off[pl.dataset[s]];
        si.n = pl.n_layers[s];
        si.nq = nq;
        si.n_chunks = std::max(1, (nq + kFp64Block - 1) / kFp64Block);
        si.part_base = slot;
        si.pad = 0;
        slot += si.n_chunks;
        for (int c = 0; c < si.n_chunks; ++c) {
            WorkItem w;
            w.stack = s;
            w.q_lo = std::min(c * kFp64Block, nq);
            w.q_hi = std::min((c + 1) * kFp64Block, nq);
            w.chunk = c;
            items.push_back(w);
        }
        maxp = std::max(maxp, 4 * si.n + 6);
        par += 4 * (int64_t)si.n + 6;
        out += nq;
    }
    pl.n64_items = (int)items.size();
    pl.n64_pert = 2 * maxp + 1;
    NR_CUDA(pl.d64_stacks.ensure(sizeof(StackInfo) * std::max(S, 1)));
    NR_CUDA(pl.d64_items.ensure(sizeof(WorkItem) * std::max<size_t>(items.size(), 1)));
    NR_CUDA(pl.d64_llpert.ensure(sizeof(double) * std::max<int64_t>(slot * pl.n64_pert, 1)));
    NR_CUDA(cudaMemcpy(pl.d64_stacks.p, info.data(), sizeof(StackInfo) * S, cudaMemcpyHostToDevice));
    if (!items.empty())
        NR_CUDA(cudaMemcpy(pl.d64_items.p, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice));
    return NR_OK;
}

nr_status get_plan(nr_ctx *ctx, const nr_batch *b, int mode, Plan **out)
{
    const int K = ctx->qc.K;
    // At most 8 cached plans, the most recently used first: the sizes and then
    // a memcmp of the host metadata decide (a mismatch usually ends early).
    // A per-call hash of the metadata cost more on the host than this scan.
    Plan *pl = nullptr;
    for (auto &p : ctx->plans)
        if (p->last_use == ctx->clock && same_meta(*p, b, K)) { pl = p.get(); break; }
    if (!pl)
        for (auto &p : ctx->plans)
            if (same_meta(*p, b, K)) { pl = p.get(); break; }
    if (!pl) {
        nr_status st = validate(b);
        if (st != NR_OK) return st;
        if (ctx->plans.size() >= 8) { // evict the least recently used plan
            auto it = std::min_element(ctx->plans.begin(), ctx->plans.end(),
                                       [](const auto &a, const auto &c) { return a->last_use < c->last_use; });
            cudaDeviceSynchronize();
            ctx->plans.erase(it);
        }
        auto np = std::make_unique<Plan>();
        np->S = b->n_stacks;
        np->D = b->n_datasets;
        np->K = K;
        if (np->S > 0) {
            np->n_layers.assign(b->n_layers, b->n_layers + np->S);
            np->dataset.assign(b->dataset, b->dataset + np->S);
            np->q_off.assign(b->q_off, b->q_off + np->D + 1);
            for (int s = 0; s < np->S; ++s) {
                const int64_t len = np->q_off[np->dataset[s] + 1] - np->q_off[np->dataset[s]];
                np->total_params += 4 * (int64_t)np->n_layers[s] + 6;
                np->total_out += len;
            }
            np->total_q = np->q_off[np->D];
            np->evals = np->total_out * K;
        }
        pl = np.get();
        ctx->plans.push_back(std::move(np));
    }
    pl->last_use = ++ctx->clock;
    if (pl->S > 0) {
        nr_status st = NR_OK;
        if (ctx->opt.precision == NR_FP64_PLAIN) {
            if (!pl->fp64_built) { st = build_fp64(ctx, *pl); pl->fp64_built = st == NR_OK; }
        } else if (is_grad_mode(mode)) {
            if (!pl->grad_built) { st = build_worklist(ctx, *pl, kGrad, pl->grad); pl->grad_built = st == NR_OK; }
        } else {
            if (!pl->fwd_built) { st = build_worklist(ctx, *pl, kModel, pl->fwd); pl->fwd_built = st == NR_OK; }
        }
        if (st != NR_OK) return st;
    }
    *out = pl;
    return NR_OK;
}

nr_status launch_device(nr_ctx *ctx, Plan &pl, const nr_batch *b, int mode, float *r_out, double *ll,
                        double *grad, double *gres, cudaStream_t st, const double *dq_scale = nullptr)
{
    if (pl.S == 0) return NR_OK;
    KernelArgs a{};
    a.dq_scale = dq_scale;
    a.params = b->params;
    a.q = b->q;
    a.dq = b->dq;
    a.r_obs = b->r_obs;
    a.r_err = b->r_err;
    a.r_out = r_out;
    a.ll_out = ll;
    a.grad_out = grad;
    a.res_out = gres;
    a.status = ctx->d_status;
    a.n_stacks = pl.S;
    if (ctx->opt.precision == NR_FP64_PLAIN) {
        a.stacks = pl.d64_stacks.as<StackInfo>();
        a.items = pl.d64_items.as<WorkItem>();
        a.n_items = pl.n64_items;
        a.ll_pert = pl.d64_llpert.as<double>();
        a.n_pert = mode == kGrad ? pl.n64_pert : 1;
        cudaError_t e = launch_fp64(mode, a, ctx->qc, st);
        if (e == cudaSuccess) e = launch_fp64_finalize(mode, pl.S, a, st);
        if (e != cudaSuccess) return fail(NR_ECUDA, "fp64 launch: %s", cudaGetErrorString(e));
        return NR_OK;
    }
    WorkList &wl = is_grad_mode(mode) ? pl.grad : pl.fwd;
    a.stacks = wl.d_stacks.as<StackInfo>();
    a.partials = wl.d_partials.as<double>();
    a.stack_done = wl.d_done.as<int32_t>();
    // Several register buckets: each is its own persistent launch; they run
    // concurrently on forked streams (joined back into `st` before the call
    // returns), so the tail of one bucket's queue overlaps the others' work
    // instead of idling SMs.  Every bucket writes disjoint outputs, partial
    // slots and tickets.  A fork / join of events is legal in stream capture.
    const size_t G_n = wl.groups.size();
    const bool fork = G_n > 1 && !ctx->opt.serial && ctx->side.size() + 1 >= G_n && ctx->ev_join.size() + 1 >= G_n;
    if (fork) NR_CUDA(cudaEventRecord(ctx->ev_fork, st));
    for (size_t g = 0; g < G_n; ++g) {
        const Group &G = wl.groups[g];
        a.items = wl.d_items.as<WorkItem>() + G.item_begin;
        a.n_items = G.item_count;
        a.tile_q = G.tile_q;
        a.ticket = wl.d_ticket.as<int32_t>() + 2 * g;
        cudaStream_t sg = st;
        if (fork && g > 0) {
            sg = ctx->side[g - 1];
            NR_CUDA(cudaStreamWaitEvent(sg, ctx->ev_fork, 0));
        }
        cudaError_t e = launch_mixed(mode, G.nmax, G.grid, a, ctx->qc, sg, G.pair);
        if (e != cudaSuccess) return fail(NR_ECUDA, "mixed launch (bucket %d): %s", G.nmax, cudaGetErrorString(e));
        if (fork && g > 0) NR_CUDA(cudaEventRecord(ctx->ev_join[g - 1], sg));
    }
    if (fork)
        for (size_t g = 1; g < G_n; ++g) NR_CUDA(cudaStreamWaitEvent(st, ctx->ev_join[g - 1], 0));
    return NR_OK;
}

// Autotuning (nr_plan on a context created with autotune = 1, device-memory
// batches, NR_MIXED): for every register bucket of a work list, time the
// candidate launch shapes on the batch's own data and keep the fastest.  The
// candidates are the paired and the one-evaluation kernel (where both apply)
// x the widest tile and half of it x the occupancy limit of CTAs per SM, one
// fewer and half of it (each a grid of that many CTAs per SM).  The work
// items (chunking) stay as planned.  Outputs go to scratch buffers; the
// device status word sees the timing launches like any call.  With
// NR_TUNE_CACHE set, a bucket whose key is in the cache file takes the
// stored shape without timing, and new choices are appended to the file.
constexpr int kTunerVersion = 2;

std::string tune_key(const nr_ctx *ctx, int mode, int nmax, int items)
{
    int lg = 0;
    while ((1 << (lg + 1)) <= items) ++lg;
    char buf[320];
    snprintf(buf, sizeof buf, "%.200s|%d|%d|%d|%d|%d|t%d", ctx->gpu_name, ctx->sms, is_grad_mode(mode) ? 2 : 0,
             ctx->qc.K, nmax, lg, kTunerVersion);
    return buf;
}

nr_status autotune_worklist(nr_ctx *ctx, Plan &pl, const nr_batch *b, bool grad)
{
    WorkList &wl = grad ? pl.grad : pl.fwd;
    if (pl.S == 0 || wl.groups.empty() || wl.tuned) return NR_OK;
    const bool lik = b->r_obs && b->r_err;
    const int mode = grad ? kGrad : (lik ? kLoglik : kModel);
    if (mode != kModel && !lik) return NR_OK;
    const int K = ctx->qc.K;
    const char *cache = std::getenv("NR_TUNE_CACHE");
    if (cache && !*cache) cache = nullptr;
    DevBuf out, ll, gr;
    if (mode == kModel) NR_CUDA(out.ensure(sizeof(float) * std::max<int64_t>(pl.total_out, 1)));
    else NR_CUDA(ll.ensure(sizeof(double) * pl.S));
    if (grad) NR_CUDA(gr.ensure(sizeof(double) * std::max<int64_t>(pl.total_params, 1)));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NR_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    KernelArgs a{};
    a.params = b->params;
    a.q = b->q;
    a.dq = b->dq;
    a.r_obs = b->r_obs;
    a.r_err = b->r_err;
    a.r_out = out.as<float>();
    a.ll_out = ll.as<double>();
    a.grad_out = gr.as<double>();
    a.status = ctx->d_status;
    a.n_stacks = pl.S;
    a.stacks = wl.d_stacks.as<StackInfo>();
    a.partials = wl.d_partials.as<double>();
    a.stack_done = wl.d_done.as<int32_t>();
    constexpr int kReps = 3;
    for (size_t g = 0; g < wl.groups.size() && ce == cudaSuccess; ++g) {
        Group &G = wl.groups[g];
        a.items = wl.d_items.as<WorkItem>() + G.item_begin;
        a.n_items = G.item_count;
        a.ticket = wl.d_ticket.as<int32_t>() + 2 * g;
        const std::string key = tune_key(ctx, mode, G.nmax, G.item_count);
        nr_tune_entry hit{};
        if (cache && nr_tune_cache_get(cache, key.c_str(), &hit) == NR_OK && hit.tile_q >= 1 &&
            hit.ctas_per_sm >= 1) {
            const bool pv = hit.paired && pair_eligible(mode, G.nmax, K);
            int tmax = mixed_tile_q(mode, G.nmax, K, pv);
            if (ctx->opt.tile_q > 0) tmax = std::min(tmax, ctx->opt.tile_q);
            int occ = 1;
            ce = mixed_occupancy(mode, G.nmax, K, &occ, pv);
            if (ce != cudaSuccess) break;
            G.pair = pv;
            G.tile_q = std::max(1, std::min(hit.tile_q, tmax));
            G.grid = std::max(1, (int)std::min<int64_t>(G.item_count,
                                                        (int64_t)ctx->sms * std::min(hit.ctas_per_sm, std::max(occ, 1))));
            continue;
        }
        float best_ms = 0.f;
        Group best = G;
        int best_ctas = 0;
        for (int pv = 1; pv >= 0 && ce == cudaSuccess; --pv) {
            if (pv == 1 && !pair_eligible(mode, G.nmax, K)) continue;
            int occ = 1;
            ce = mixed_occupancy(mode, G.nmax, K, &occ, pv == 1);
            if (ce != cudaSuccess) break;
            occ = std::max(occ, 1);
            int tmax = mixed_tile_q(mode, G.nmax, K, pv == 1);
            if (ctx->opt.tile_q > 0) tmax = std::min(tmax, ctx->opt.tile_q);
            tmax = std::max(tmax, 1);
            int cands[3] = {occ, occ - 1, (occ + 1) / 2};
            for (int ci = 0; ci < 3 && ce == cudaSuccess; ++ci) {
                const int cps = cands[ci];
                if (cps < 1 || (ci > 0 && cps == cands[0]) || (ci == 2 && cps == cands[1])) continue;
                int grid = (int)std::min<int64_t>(G.item_count, (int64_t)ctx->sms * cps);
                if (ctx->opt.grid_ctas > 0) grid = std::min(G.item_count, ctx->opt.grid_ctas);
                grid = std::max(grid, 1);
                for (int tq : {tmax, tmax / 2}) {
                    if (tq < 1) continue;
                    a.tile_q = tq;
                    ce = launch_mixed(mode, G.nmax, grid, a, ctx->qc, st, pv == 1); // warm-up
                    if (ce == cudaSuccess) ce = cudaEventRecord(e0, st);
                    for (int r = 0; r < kReps && ce == cudaSuccess; ++r)
                        ce = launch_mixed(mode, G.nmax, grid, a, ctx->qc, st, pv == 1);
                    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
                    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                    float ms = 0.f;
                    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                    if (ce != cudaSuccess) break;
                    if (best_ms == 0.f || ms < best_ms) {
                        best_ms = ms;
                        best.pair = pv == 1;
                        best.tile_q = tq;
                        best.grid = grid;
                        best_ctas = cps;
                    }
                }
            }
        }
        if (ce == cudaSuccess) {
            G = best;
            if (cache) {
                nr_tune_entry e{};
                e.paired = best.pair ? 1 : 0;
                e.tile_q = best.tile_q;
                e.ctas_per_sm = best_ctas;
                e.ms = best_ms / kReps;
                nr_tune_cache_put(cache, key.c_str(), &e); // best effort: a read-only cache still tunes
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const cudaError_t se = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (ce == cudaSuccess) ce = se;
    if (ce != cudaSuccess) return fail(NR_ECUDA, "autotune: %s", cudaGetErrorString(ce));
    wl.tuned = true;
    return NR_OK;
}

// Host-memory batches: copy in, compute, copy out, synchronise.
nr_status run_host(nr_ctx *ctx, Plan &pl, const nr_batch *b, int mode, float *r_out, double *ll, double *grad,
                   double *gres, cudaStream_t st)
{
    if (pl.S == 0) return NR_OK;
    const size_t np = sizeof(double) * pl.total_params, nqb = sizeof(float) * pl.total_q;
    const bool need_data = mode != kModel;
    NR_CUDA(ctx->s_params.ensure(np));
    NR_CUDA(ctx->s_q.ensure(nqb));
    NR_CUDA(ctx->s_dq.ensure(nqb));
    if (need_data) {
        if (!b->r_obs || !b->r_err) return fail(NR_EINVAL, "r_obs/r_err required");
        NR_CUDA(ctx->s_robs.ensure(nqb));
        NR_CUDA(ctx->s_rerr.ensure(nqb));
    }
    NR_CUDA(cudaMemcpyAsync(ctx->s_params.p, b->params, np, cudaMemcpyHostToDevice, st));
    NR_CUDA(cudaMemcpyAsync(ctx->s_q.p, b->q, nqb, cudaMemcpyHostToDevice, st));
    NR_CUDA(cudaMemcpyAsync(ctx->s_dq.p, b->dq, nqb, cudaMemcpyHostToDevice, st));
    if (need_data) {
        NR_CUDA(cudaMemcpyAsync(ctx->s_robs.p, b->r_obs, nqb, cudaMemcpyHostToDevice, st));
        NR_CUDA(cudaMemcpyAsync(ctx->s_rerr.p, b->r_err, nqb, cudaMemcpyHostToDevice, st));
    }
    nr_batch db = *b;
    db.memory = NR_MEM_DEVICE;
    db.params = ctx->s_params.as<double>();
    db.q = ctx->s_q.as<float>();
    db.dq = ctx->s_dq.as<float>();
    db.r_obs = need_data ? ctx->s_robs.as<float>() : nullptr;
    db.r_err = need_data ? ctx->s_rerr.as<float>() : nullptr;
    float *d_out = nullptr;
    double *d_ll = nullptr, *d_grad = nullptr, *d_res = nullptr;
    if (r_out) { NR_CUDA(ctx->s_out.ensure(sizeof(float) * pl.total_out)); d_out = ctx->s_out.as<float>(); }
    if (ll) { NR_CUDA(ctx->s_ll.ensure(sizeof(double) * pl.S)); d_ll = ctx->s_ll.as<double>(); }
    if (grad) { NR_CUDA(ctx->s_grad.ensure(np)); d_grad = ctx->s_grad.as<double>(); }
    if (gres) { NR_CUDA(ctx->s_res.ensure(sizeof(double) * pl.S)); d_res = ctx->s_res.as<double>(); }
    nr_status s = launch_device(ctx, pl, &db, mode, d_out, d_ll, d_grad, d_res, st);
    if (s != NR_OK) return s;
    if (r_out) NR_CUDA(cudaMemcpyAsync(r_out, d_out, sizeof(float) * pl.total_out, cudaMemcpyDeviceToHost, st));
    if (ll) NR_CUDA(cudaMemcpyAsync(ll, d_ll, sizeof(double) * pl.S, cudaMemcpyDeviceToHost, st));
    if (grad) NR_CUDA(cudaMemcpyAsync(grad, d_grad, np, cudaMemcpyDeviceToHost, st));
    if (gres) NR_CUDA(cudaMemcpyAsync(gres, d_res, sizeof(double) * pl.S, cudaMemcpyDeviceToHost, st));
    NR_CUDA(cudaStreamSynchronize(st));
    return NR_OK;
}

nr_status compute(nr_ctx *ctx, const nr_batch *b, int mode, float *r_out, double *ll, double *grad, double *gres,
                  void *stream, const double *dq_scale = nullptr)
{
    static const char *const kNames[] = {"nr_reflectivity", "nr_loglik", "nr_loglik_grad", "nr_loglik_grad_res"};
    NvtxRange range(kNames[mode]);
    if (!ctx) return fail(NR_EINVAL, "context is NULL");
    if (!b) return fail(NR_EINVAL, "batch is NULL");
    if (mode == kModel && !r_out && b->n_stacks > 0) return fail(NR_EINVAL, "r_out is NULL");
    if (mode == kLoglik && !ll && b->n_stacks > 0) return fail(NR_EINVAL, "loglik is NULL");
    if (mode != kModel && b->n_stacks > 0 && (!b->r_obs || !b->r_err))
        return fail(NR_EINVAL, "r_obs/r_err are required for the likelihood");
    if (mode == kGradRes && ctx->opt.precision != NR_MIXED)
        return fail(NR_EINVAL, "the resolution derivative is computed by the NR_MIXED path only");
    NR_CUDA(cudaSetDevice(ctx->device));
    Plan *pl = nullptr;
    nr_status st = get_plan(ctx, b, mode, &pl);
    if (st != NR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->memory == NR_MEM_HOST) return run_host(ctx, *pl, b, mode, r_out, ll, grad, gres, s);
    return launch_device(ctx, *pl, b, mode, r_out, ll, grad, gres, s, dq_scale);
}

} // namespace

// ================================================================ C ABI ===
extern "C" {

nr_status nr_create(nr_ctx **out, const nr_options *opt)
{
    if (!out) return fail(NR_EINVAL, "out is NULL");
    *out = nullptr;
    auto ctx = std::make_unique<nr_ctx>();
    ctx->opt.n_quad = 17;
    ctx->opt.precision = NR_MIXED;
    ctx->opt.deterministic = 1;
    if (opt) {
        ctx->opt = *opt;
        if (ctx->opt.n_quad == 0) ctx->opt.n_quad = 17;
    }
    if (ctx->opt.n_quad < 1 || ctx->opt.n_quad > NR_MAX_QUAD)
        return fail(NR_EINVAL, "n_quad %d outside [1, %d]", ctx->opt.n_quad, NR_MAX_QUAD);
    if (ctx->opt.precision != NR_MIXED && ctx->opt.precision != NR_FP64_PLAIN)
        return fail(NR_EINVAL, "unknown precision %d", ctx->opt.precision);
    if (ctx->opt.tile_q < 0 || ctx->opt.chunk_q < 0 || ctx->opt.grid_ctas < 0)
        return fail(NR_EINVAL, "negative launch override");
    if (!make_quad_const(ctx->opt.n_quad, ctx->qc)) return fail(NR_EINVAL, "quadrature failed");
    NR_CUDA(cudaGetDevice(&ctx->device));
    NR_CUDA(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device));
    {
        cudaDeviceProp prop{};
        NR_CUDA(cudaGetDeviceProperties(&prop, ctx->device));
        snprintf(ctx->gpu_name, sizeof ctx->gpu_name, "%s", prop.name);
        for (char *c = ctx->gpu_name; *c; ++c)
            if (*c == '"' || *c == '\\' || *c == '|') *c = '_';
    }
    NR_CUDA(dev_malloc(reinterpret_cast<void **>(&ctx->d_status), sizeof(int32_t)));
    NR_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    *out = ctx.release();
    return NR_OK;
}

void nr_destroy(nr_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->d_status) cudaFree(ctx->d_status);
    for (cudaStream_t s : ctx->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : ctx->ev_join) cudaEventDestroy(e);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    delete ctx;
}

const char *nr_last_error(void) { return g_last_error.c_str(); }

nr_status nr_plan(nr_ctx *ctx, const nr_batch *batch)
{
    if (!ctx) return fail(NR_EINVAL, "context is NULL");
    NR_CUDA(cudaSetDevice(ctx->device));
    Plan *pl = nullptr;
    nr_status st = get_plan(ctx, batch, kModel, &pl);
    if (st == NR_OK) st = get_plan(ctx, batch, kGrad, &pl);
    if (st == NR_OK && ctx->opt.autotune && ctx->opt.precision == NR_MIXED && batch->memory == NR_MEM_DEVICE) {
        st = autotune_worklist(ctx, *pl, batch, false);
        if (st == NR_OK) st = autotune_worklist(ctx, *pl, batch, true);
    }
    return st;
}

nr_status nr_reflectivity(nr_ctx *ctx, const nr_batch *batch, float *r_out, void *stream)
{
    return compute(ctx, batch, kModel, r_out, nullptr, nullptr, nullptr, stream);
}

nr_status nr_loglik(nr_ctx *ctx, const nr_batch *batch, double *loglik, void *stream)
{
    return compute(ctx, batch, kLoglik, nullptr, loglik, nullptr, nullptr, stream);
}

nr_status nr_loglik_grad(nr_ctx *ctx, const nr_batch *batch, double *loglik, double *grad, void *stream)
{
    return compute(ctx, batch, kGrad, nullptr, loglik, grad, nullptr, stream);
}

nr_status nr_loglik_grad_res(nr_ctx *ctx, const nr_batch *batch, double *loglik, double *grad, double *grad_res,
                             void *stream)
{
    return compute(ctx, batch, kGradRes, nullptr, loglik, grad, grad_res, stream);
}

nr_status nr_sld_profile(nr_ctx *ctx, const nr_batch *batch, const float *z, int32_t nz, float *rho_out,
                         float *iota_out, void *stream)
{
    if (!ctx) return fail(NR_EINVAL, "context is NULL");
    if (!batch) return fail(NR_EINVAL, "batch is NULL");
    const nr_batch *b = batch;
    if (b->n_stacks < 0) return fail(NR_EINVAL, "n_stacks < 0");
    if (b->memory != NR_MEM_DEVICE && b->memory != NR_MEM_HOST) return fail(NR_EINVAL, "bad memory kind");
    if (nz < 0) return fail(NR_EINVAL, "nz < 0");
    const int S = b->n_stacks;
    if (S == 0 || nz == 0) return NR_OK;
    if (!b->n_layers || !b->params) return fail(NR_EINVAL, "n_layers/params pointer is NULL");
    if (!z) return fail(NR_EINVAL, "z is NULL");
    if (!rho_out && !iota_out) return fail(NR_EINVAL, "rho_out and iota_out are both NULL");
    std::vector<int64_t> off(S);
    int64_t np = 0;
    for (int s = 0; s < S; ++s) {
        if (b->n_layers[s] < 0 || b->n_layers[s] > NR_MAX_LAYERS)
            return fail(NR_EINVAL, "stack %d: n_layers %d outside [0, %d]", s, b->n_layers[s], NR_MAX_LAYERS);
        off[s] = np;
        np += 4 * (int64_t)b->n_layers[s] + 6;
    }
    NR_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    NR_CUDA(ctx->p_off.ensure(sizeof(int64_t) * S));
    NR_CUDA(ctx->p_nl.ensure(sizeof(int32_t) * S));
    NR_CUDA(cudaMemcpyAsync(ctx->p_off.p, off.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, st));
    NR_CUDA(cudaMemcpyAsync(ctx->p_nl.p, b->n_layers, sizeof(int32_t) * S, cudaMemcpyHostToDevice, st));
    const size_t nout = sizeof(float) * (size_t)S * nz;
    const double *d_par = b->params;
    const float *d_z = z;
    float *d_rho = rho_out, *d_iota = iota_out;
    if (b->memory == NR_MEM_HOST) {
        NR_CUDA(ctx->s_params.ensure(sizeof(double) * np));
        NR_CUDA(ctx->p_z.ensure(sizeof(float) * nz));
        NR_CUDA(cudaMemcpyAsync(ctx->s_params.p, b->params, sizeof(double) * np, cudaMemcpyHostToDevice, st));
        NR_CUDA(cudaMemcpyAsync(ctx->p_z.p, z, sizeof(float) * nz, cudaMemcpyHostToDevice, st));
        d_par = ctx->s_params.as<double>();
        d_z = ctx->p_z.as<float>();
        if (rho_out) { NR_CUDA(ctx->p_rho.ensure(nout)); d_rho = ctx->p_rho.as<float>(); }
        if (iota_out) { NR_CUDA(ctx->p_iota.ensure(nout)); d_iota = ctx->p_iota.as<float>(); }
    }
    cudaError_t e = launch_profile(d_par, ctx->p_off.as<int64_t>(), ctx->p_nl.as<int32_t>(), S, d_z, nz, d_rho,
                                   d_iota, ctx->d_status, ctx->sms, st);
    if (e != cudaSuccess) return fail(NR_ECUDA, "profile launch: %s", cudaGetErrorString(e));
    if (b->memory == NR_MEM_HOST) {
        if (rho_out) NR_CUDA(cudaMemcpyAsync(rho_out, d_rho, nout, cudaMemcpyDeviceToHost, st));
        if (iota_out) NR_CUDA(cudaMemcpyAsync(iota_out, d_iota, nout, cudaMemcpyDeviceToHost, st));
        NR_CUDA(cudaStreamSynchronize(st));
    }
    return NR_OK;
}

nr_status nr_sampler_create(nr_ctx *ctx, const nr_cofit_model *m, nr_sampler **out)
{
    if (!out) return fail(NR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctx || !m) return fail(NR_EINVAL, "context or model is NULL");
    if (ctx->opt.precision != NR_MIXED) return fail(NR_EINVAL, "the samplers run on the NR_MIXED path");
    if (m->n_chains < 1 || m->n_contrasts < 1 || m->n_free < 1) return fail(NR_EINVAL, "empty model");
    if ((int64_t)m->n_chains * m->n_contrasts > (int64_t)1 << 30) return fail(NR_EINVAL, "model too large");
    if (!m->n_layers || !m->dataset || !m->q_off || !m->slot_src || !m->slot_val || !m->lo || !m->hi)
        return fail(NR_EINVAL, "model host pointer is NULL");
    if (!m->q || !m->dq || !m->r_obs || !m->r_err) return fail(NR_EINVAL, "model data pointer is NULL");
    const int C = m->n_chains, NC = m->n_contrasts, P = m->n_free;
    int NS = 0;
    for (int c = 0; c < NC; ++c) {
        if (m->n_layers[c] < 0 || m->n_layers[c] > NR_MAX_LAYERS)
            return fail(NR_EINVAL, "contrast %d: n_layers %d outside [0, %d]", c, m->n_layers[c], NR_MAX_LAYERS);
        NS += 4 * m->n_layers[c] + 6;
    }
    for (int k = 0; k < P; ++k)
        if (!std::isfinite(m->lo[k]) || !std::isfinite(m->hi[k]) || !(m->lo[k] < m->hi[k]))
            return fail(NR_EINVAL, "parameter %d: bounds [%g, %g]", k, m->lo[k], m->hi[k]);
    if (m->res_param < -1 || m->res_param >= P)
        return fail(NR_EINVAL, "res_param %d outside [-1, %d)", m->res_param, P);
    if (m->res_param >= 0 && !(m->lo[m->res_param] > 0.0))
        return fail(NR_EINVAL, "resolution scale parameter %d: lower bound %g not positive", m->res_param,
                    m->lo[m->res_param]);
    std::vector<int32_t> tie_ptr(P + 1, 0), tie_slot;
    for (int i = 0; i < NS; ++i) {
        const int k = m->slot_src[i];
        if (k < -1 || k >= P) return fail(NR_EINVAL, "slot %d: source %d outside [-1, %d)", i, k, P);
        if (k < 0 && !std::isfinite(m->slot_val[i])) return fail(NR_EINVAL, "slot %d: fixed value not finite", i);
        if (k >= 0) ++tie_ptr[k + 1];
    }
    for (int k = 0; k < P; ++k) tie_ptr[k + 1] += tie_ptr[k];
    tie_slot.resize(std::max(tie_ptr[P], 1));
    {
        std::vector<int32_t> fill(tie_ptr.begin(), tie_ptr.end() - 1);
        for (int i = 0; i < NS; ++i)
            if (m->slot_src[i] >= 0) tie_slot[fill[m->slot_src[i]]++] = i;
    }
    auto sp = std::make_unique<nr_sampler>();
    nr_sampler &S = *sp;
    S.ctx = ctx;
    S.device = ctx->device;
    S.C = C;
    S.P = P;
    S.NC = NC;
    S.NS = NS;
    S.n_layers.resize((size_t)C * NC);
    S.dataset.resize((size_t)C * NC);
    for (int c = 0; c < C; ++c)
        for (int j = 0; j < NC; ++j) {
            S.n_layers[(size_t)c * NC + j] = m->n_layers[j];
            S.dataset[(size_t)c * NC + j] = m->dataset[j];
        }
    if (m->n_datasets < 1) return fail(NR_EINVAL, "n_datasets < 1");
    S.q_off.assign(m->q_off, m->q_off + m->n_datasets + 1);
    NR_CUDA(cudaSetDevice(ctx->device));
    NR_CUDA(S.d_src.ensure(sizeof(int32_t) * NS));
    NR_CUDA(S.d_val.ensure(sizeof(double) * NS));
    NR_CUDA(S.d_lo.ensure(sizeof(double) * P));
    NR_CUDA(S.d_hi.ensure(sizeof(double) * P));
    NR_CUDA(S.d_tie_ptr.ensure(sizeof(int32_t) * (P + 1)));
    NR_CUDA(S.d_tie_slot.ensure(sizeof(int32_t) * tie_slot.size()));
    NR_CUDA(S.d_params.ensure(sizeof(double) * (size_t)C * NS));
    NR_CUDA(S.d_ll.ensure(sizeof(double) * (size_t)C * NC));
    NR_CUDA(S.d_gpk.ensure(sizeof(double) * (size_t)C * NS));
    NR_CUDA(S.d_mom.ensure(sizeof(double) * (size_t)C * P));
    NR_CUDA(S.d_u0.ensure(sizeof(double) * (size_t)C * P));
    NR_CUDA(S.d_H0.ensure(sizeof(double) * C));
    NR_CUDA(S.d_lp0.ensure(sizeof(double) * C));
    NR_CUDA(S.d_vu.ensure(sizeof(double) * (size_t)C * P));
    NR_CUDA(S.d_vg.ensure(sizeof(double) * (size_t)C * P));
    NR_CUDA(S.d_vlp.ensure(sizeof(double) * C));
    NR_CUDA(S.d_vpart.ensure(sizeof(double) * C));
    NR_CUDA(S.d_vbias.ensure(sizeof(double) * 2));
    S.res_param = m->res_param;
    if (S.res_param >= 0) {
        NR_CUDA(S.d_dqs.ensure(sizeof(double) * (size_t)C * NC));
        NR_CUDA(S.d_gres.ensure(sizeof(double) * (size_t)C * NC));
    }
    NR_CUDA(cudaMemcpy(S.d_src.p, m->slot_src, sizeof(int32_t) * NS, cudaMemcpyHostToDevice));
    NR_CUDA(cudaMemcpy(S.d_val.p, m->slot_val, sizeof(double) * NS, cudaMemcpyHostToDevice));
    NR_CUDA(cudaMemcpy(S.d_lo.p, m->lo, sizeof(double) * P, cudaMemcpyHostToDevice));
    NR_CUDA(cudaMemcpy(S.d_hi.p, m->hi, sizeof(double) * P, cudaMemcpyHostToDevice));
    NR_CUDA(cudaMemcpy(S.d_tie_ptr.p, tie_ptr.data(), sizeof(int32_t) * (P + 1), cudaMemcpyHostToDevice));
    NR_CUDA(cudaMemcpy(S.d_tie_slot.p, tie_slot.data(), sizeof(int32_t) * tie_slot.size(), cudaMemcpyHostToDevice));
    // fixed slots in place from the start (tied ones are rewritten by every gather)
    for (int c = 0; c < C; ++c)
        NR_CUDA(cudaMemcpy(S.d_params.as<double>() + (size_t)c * NS, m->slot_val, sizeof(double) * NS,
                           cudaMemcpyHostToDevice));
    nr_batch &b = S.batch;
    b.n_stacks = C * NC;
    b.n_datasets = m->n_datasets;
    b.n_layers = S.n_layers.data();
    b.dataset = S.dataset.data();
    b.q_off = S.q_off.data();
    b.memory = NR_MEM_DEVICE;
    b.params = S.d_params.as<double>();
    b.q = m->q;
    b.dq = m->dq;
    b.r_obs = m->r_obs;
    b.r_err = m->r_err;
    Plan *pl = nullptr;
    nr_status st = get_plan(ctx, &b, kGrad, &pl);
    if (st != NR_OK) return st;
    *out = sp.release();
    return NR_OK;
}

void nr_sampler_destroy(nr_sampler *s)
{
    if (!s) return;
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    delete s;
}

namespace {
CofitStageArgs stage_args(nr_sampler *S, double *u, int stage)
{
    CofitStageArgs a{};
    a.C = S->C;
    a.P = S->P;
    a.NS = S->NS;
    a.n_contrast = S->NC;
    a.stage = stage;
    a.u = u;
    a.ll = S->d_ll.as<double>();
    a.gpk = S->d_gpk.as<double>();
    a.tie_ptr = S->d_tie_ptr.as<int32_t>();
    a.tie_slot = S->d_tie_slot.as<int32_t>();
    a.lo = S->d_lo.as<double>();
    a.hi = S->d_hi.as<double>();
    a.mom = S->d_mom.as<double>();
    a.u0 = S->d_u0.as<double>();
    a.H0 = S->d_H0.as<double>();
    a.logp0 = S->d_lp0.as<double>();
    a.res_param = S->res_param;
    a.gres = S->d_gres.as<double>();
    return a;
}

// log-likelihood and packed gradient of every stack at the chains' u
nr_status sampler_eval(nr_sampler *S, const double *u, cudaStream_t st)
{
    cudaError_t e = launch_cofit_gather(u, S->C, S->P, S->NS, S->d_src.as<int32_t>(), S->d_val.as<double>(),
                                        S->d_lo.as<double>(), S->d_hi.as<double>(), S->d_params.as<double>(),
                                        S->res_param, S->NC, S->d_dqs.as<double>(), st);
    if (e != cudaSuccess) return fail(NR_ECUDA, "sampler gather: %s", cudaGetErrorString(e));
    if (S->res_param >= 0)
        return compute(S->ctx, &S->batch, kGradRes, nullptr, S->d_ll.as<double>(), S->d_gpk.as<double>(),
                       S->d_gres.as<double>(), st, S->d_dqs.as<double>());
    return compute(S->ctx, &S->batch, kGrad, nullptr, S->d_ll.as<double>(), S->d_gpk.as<double>(), nullptr, st);
}
} // namespace

nr_status nr_sampler_logp_grad(nr_sampler *S, const double *u, double *logp, double *grad, void *stream)
{
    if (!S || !u) return fail(NR_EINVAL, "sampler or u is NULL");
    NR_CUDA(cudaSetDevice(S->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    nr_status r = sampler_eval(S, u, st);
    if (r != NR_OK) return r;
    CofitStageArgs a = stage_args(S, const_cast<double *>(u), kStageLogp);
    a.logp_out = logp;
    a.grad_out = grad;
    cudaError_t e = launch_cofit_stage(a, st);
    if (e != cudaSuccess) return fail(NR_ECUDA, "sampler stage: %s", cudaGetErrorString(e));
    return NR_OK;
}

nr_status nr_hmc_step(nr_sampler *S, double *u, const double *z, const double *log_unif, const double *inv_mass,
                      double eps, int32_t n_leapfrog, double *logp, int32_t *accepted, void *stream)
{
    if (!S || !u || !z || !log_unif || !inv_mass) return fail(NR_EINVAL, "sampler or array pointer is NULL");
    if (n_leapfrog < 1) return fail(NR_EINVAL, "n_leapfrog %d < 1", n_leapfrog);
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(NR_EINVAL, "step %g not positive", eps);
    NR_CUDA(cudaSetDevice(S->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int l = 0; l <= n_leapfrog; ++l) {
        nr_status r = sampler_eval(S, u, st);
        if (r != NR_OK) return r;
        CofitStageArgs a = stage_args(S, u, l == 0 ? kStageFirst : l == n_leapfrog ? kStageLast : kStageMid);
        a.eps = eps;
        a.inv_mass = inv_mass;
        a.z = z;
        a.log_unif = log_unif;
        a.logp_out = logp;
        a.accepted = accepted;
        cudaError_t e = launch_cofit_stage(a, st);
        if (e != cudaSuccess) return fail(NR_ECUDA, "sampler stage: %s", cudaGetErrorString(e));
    }
    return NR_OK;
}

nr_status nr_vi_step(nr_sampler *S, double *phi, double *adam_m, double *adam_v, int32_t *t, const double *eps,
                     const nr_adam *opt, double *elbo, void *stream)
{
    if (!S || !phi || !adam_m || !adam_v || !t || !eps || !opt) return fail(NR_EINVAL, "NULL argument");
    if (!(opt->lr > 0.0) || !(opt->beta1 >= 0.0 && opt->beta1 < 1.0) || !(opt->beta2 >= 0.0 && opt->beta2 < 1.0) ||
        !(opt->eps > 0.0))
        return fail(NR_EINVAL, "Adam settings lr %g beta1 %g beta2 %g eps %g", opt->lr, opt->beta1, opt->beta2,
                    opt->eps);
    NR_CUDA(cudaSetDevice(S->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *u = S->d_vu.as<double>();
    cudaError_t e = launch_vi_sample(phi, eps, S->C, S->P, u, S->d_vpart.as<double>(), t, opt->beta1, opt->beta2,
                                     S->d_vbias.as<double>(), st);
    if (e != cudaSuccess) return fail(NR_ECUDA, "vi sample: %s", cudaGetErrorString(e));
    nr_status r = sampler_eval(S, u, st);
    if (r != NR_OK) return r;
    CofitStageArgs a = stage_args(S, u, kStageLogp);
    a.logp_out = S->d_vlp.as<double>();
    a.grad_out = S->d_vg.as<double>();
    e = launch_cofit_stage(a, st);
    if (e == cudaSuccess)
        e = launch_vi_adam(phi, adam_m, adam_v, eps, S->d_vg.as<double>(), S->d_vlp.as<double>(),
                           S->d_vpart.as<double>(), S->C, S->P, S->d_vbias.as<double>(), opt->lr, opt->beta1,
                           opt->beta2, opt->eps, elbo,
                           st);
    if (e != cudaSuccess) return fail(NR_ECUDA, "vi step: %s", cudaGetErrorString(e));
    return NR_OK;
}

nr_status nr_device_status(nr_ctx *ctx, void *stream, int32_t *flags)
{
    if (!ctx) return fail(NR_EINVAL, "context is NULL");
    NR_CUDA(cudaSetDevice(ctx->device));
    NR_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int32_t f = 0;
    NR_CUDA(cudaMemcpy(&f, ctx->d_status, sizeof f, cudaMemcpyDeviceToHost));
    NR_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    if (flags) *flags = f;
    return f ? fail(NR_ENONFINITE, "device status flags 0x%x", f) : NR_OK;
}

nr_status nr_quadrature(int32_t K, double *x, double *w)
{
    if (!x || !w) return fail(NR_EINVAL, "x/w is NULL");
    if (!gauss_hermite(K, x, w)) return fail(NR_EINVAL, "K %d outside [1, %d]", K, NR_MAX_QUAD);
    return NR_OK;
}

nr_status nr_plan_info(nr_ctx *ctx, const nr_batch *batch, int64_t *evals, int32_t *tile_q, int32_t *chunk_q,
                       int32_t *grid_ctas, int32_t *launches)
{
    if (!ctx) return fail(NR_EINVAL, "context is NULL");
    NR_CUDA(cudaSetDevice(ctx->device));
    Plan *pl = nullptr;
    nr_status st = get_plan(ctx, batch, kGrad, &pl);
    if (st != NR_OK) return st;
    if (evals) *evals = pl->evals;
    const bool fp64 = ctx->opt.precision == NR_FP64_PLAIN;
    const WorkList &wl = pl->grad;
    if (tile_q) *tile_q = fp64 ? kFp64Block : (wl.groups.empty() ? 0 : wl.groups[0].tile_q);
    if (chunk_q) *chunk_q = fp64 ? kFp64Block : wl.chunk_q;
    if (grid_ctas) *grid_ctas = fp64 ? pl->n64_items : (wl.groups.empty() ? 0 : wl.groups[0].grid);
    if (launches) *launches = fp64 ? 2 : (int32_t)wl.groups.size();
    return NR_OK;
}

nr_status nr_debug_fail_allocs(int32_t count)
{
    if (count < 0) return fail(NR_EINVAL, "count < 0");
    g_fail_allocs.store(count);
    return NR_OK;
}

nr_status nr_debug_poison_plan(nr_ctx *ctx, const nr_batch *batch, int32_t on)
{
    if (!NR_DEBUG) return fail(NR_EINVAL, "nr_debug_poison_plan needs a library built with NR_DEBUG");
    if (!ctx) return fail(NR_EINVAL, "context is NULL");
    if (on != 0 && on != 1) return fail(NR_EINVAL, "on must be 0 or 1");
    if (ctx->opt.precision != NR_MIXED) return fail(NR_EINVAL, "the hook corrupts NR_MIXED plans only");
    nr_status st = validate(batch);
    if (st != NR_OK) return st;
    if (batch->memory != NR_MEM_DEVICE) return fail(NR_EINVAL, "the hook takes a device batch");
    NR_CUDA(cudaSetDevice(ctx->device));
    Plan *pl = nullptr;
    st = get_plan(ctx, batch, kGrad, &pl);
    if (st != NR_OK) return st;
    WorkList &wl = pl->grad;
    if (wl.groups.empty() || wl.groups[0].item_count < 1) return fail(NR_EINVAL, "the plan has no work item");
    WorkItem *d_first = wl.d_items.as<WorkItem>();
    NR_CUDA(cudaDeviceSynchronize());
    if (on) {
        if (ctx->poisoned.stack >= 0) return fail(NR_EINVAL, "the plan is already poisoned");
        NR_CUDA(cudaMemcpy(&ctx->poisoned, d_first, sizeof(WorkItem), cudaMemcpyDeviceToHost));
        WorkItem bad = ctx->poisoned;
        bad.stack = pl->S;
        NR_CUDA(cudaMemcpy(d_first, &bad, sizeof(WorkItem), cudaMemcpyHostToDevice));
    } else {
        if (ctx->poisoned.stack < 0) return fail(NR_EINVAL, "the plan is not poisoned");
        NR_CUDA(cudaMemcpy(d_first, &ctx->poisoned, sizeof(WorkItem), cudaMemcpyHostToDevice));
        NR_CUDA(cudaMemset(wl.d_done.p, 0, wl.d_done.bytes));
        ctx->poisoned.stack = -1;
    }
    return NR_OK;
}

nr_status nr_plan_groups(nr_ctx *ctx, const nr_batch *batch, int32_t grad, int32_t max_groups, int32_t *count,
                         int32_t *nmax, int32_t *paired, int32_t *tile_q, int32_t *grid, int32_t *items)
{
    if (!ctx) return fail(NR_EINVAL, "context is NULL");
    if (max_groups < 0) return fail(NR_EINVAL, "max_groups < 0");
    if (ctx->opt.precision != NR_MIXED) return fail(NR_EINVAL, "launch groups exist for NR_MIXED contexts only");
    NR_CUDA(cudaSetDevice(ctx->device));
    Plan *pl = nullptr;
    nr_status st = get_plan(ctx, batch, grad ? kGrad : kModel, &pl);
    if (st != NR_OK) return st;
    const WorkList &wl = grad ? pl->grad : pl->fwd;
    if (count) *count = (int32_t)wl.groups.size();
    for (int i = 0; i < (int)wl.groups.size() && i < max_groups; ++i) {
        const Group &G = wl.groups[i];
        if (nmax) nmax[i] = G.nmax;
        if (paired) paired[i] = G.pair && pair_eligible(grad ? kGrad : kLoglik, G.nmax, ctx->qc.K) ? 1 : 0;
        if (tile_q) tile_q[i] = G.tile_q;
        if (grid) grid[i] = G.grid;
        if (items) items[i] = G.item_count;
    }
    return NR_OK;
}

} // extern "C"
