// nr_noalloc.cu -- nr_loglik_grad_noalloc: the log-likelihood + gradient
// call for callers that are not allowed to allocate device memory.
//
// Some hosts cannot let a library call cudaMalloc: a plug-in whose host
// application owns every device allocation through its own pool, a
// hard-real-time control loop that must not hit the driver's allocator, or a
// process that has already reserved nearly all of the GPU's memory.  The
// regular entry points need a context (nr_create allocates a status word) and
// a plan (device work lists).  This entry point needs neither: the work list,
// the queue tickets and the status word live in one file-scope device array
// of fixed size that every GPU loading the library holds until the process
// exits, and the caller passes only inputs and outputs.
//
// The computation is the regular mixed-precision gradient kernel (the paired
// two-evaluations-per-thread kernel wherever nr_loglik_grad uses it),
// launched once per layer bucket with one work item per stack (no chunking).
// The work list is built on the host in static arrays and copied from that
// pageable memory, so the call waits for the stream's earlier work before it
// returns; the kernels then run asynchronously.  It cannot be captured in a
// CUDA graph (refused with NR_EINVAL): a replay would copy whatever the last
// eager call left in the host arrays.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "nr.h"
#include "nr_internal.h"

namespace nrimpl {
void record_error(const char *msg); // nr_api.cpp: message for nr_last_error()
}

using namespace nrimpl;

namespace {

constexpr int kMaxStacks = NR_NOALLOC_MAX_STACKS;
constexpr int kBuckets[] = {1, 2, 4, 8, 12, 16, 20, 32, 64};
constexpr int kNumBuckets = sizeof(kBuckets) / sizeof(kBuckets[0]);
constexpr size_t kCtrlBytes = 256; // tickets (2 per bucket) and the status word
constexpr size_t kScratchBytes = kCtrlBytes + (size_t)kMaxStacks * (sizeof(StackInfo) + sizeof(WorkItem));

// The shared scratch of every nr_loglik_grad_noalloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host staging of the work list (static storage, not heap) and the device
// address of the scratch per device, looked up once with that device current.
StackInfo h_stacks[kMaxStacks];
WorkItem h_items[kMaxStacks];
int h_order[kMaxStacks];
void *g_scratch_dev[64];
std::mutex g_mutex;

nr_status err(nr_status st, const char *what)
{
    record_error(what);
    return st;
}

int bucket_of(int n)
{
    if (n == 1) return 0;
    for (int b = 1; b < kNumBuckets; ++b)
        if (n <= kBuckets[b]) return b;
    return -1;
}

} // namespace

extern "C" nr_status nr_loglik_grad_noalloc(const nr_batch *b, int32_t n_quad, double *loglik, double *grad,
                                            int32_t *device_flags, void *stream)
{
    if (!b) return err(NR_EINVAL, "batch is NULL");
    if (b->memory != NR_MEM_DEVICE) return err(NR_EINVAL, "nr_loglik_grad_noalloc takes device-memory batches only");
    if (n_quad < 1 || n_quad > NR_MAX_QUAD) return err(NR_EINVAL, "n_quad outside [1, NR_MAX_QUAD]");
    if (b->n_stacks < 0) return err(NR_EINVAL, "n_stacks < 0");
    if (b->n_stacks > kMaxStacks) {
        char msg[160];
        snprintf(msg, sizeof msg, "n_stacks %d exceeds the no-allocation limit NR_NOALLOC_MAX_STACKS = %d",
                 b->n_stacks, kMaxStacks);
        return err(NR_EINVAL, msg);
    }
    if (b->n_stacks == 0) return NR_OK;
    const int S = b->n_stacks;
    if (b->n_datasets < 1 || !b->n_layers || !b->dataset || !b->q_off) return err(NR_EINVAL, "bad metadata");
    if (!b->params || !b->q || !b->dq || !b->r_obs || !b->r_err) return err(NR_EINVAL, "a bulk pointer is NULL");
    if (b->q_off[0] != 0) return err(NR_EINVAL, "q_off[0] != 0");
    for (int d = 0; d < b->n_datasets; ++d) {
        const int64_t len = b->q_off[d + 1] - b->q_off[d];
        if (len < 0 || len > (int64_t)1 << 30) return err(NR_EINVAL, "q_off not non-decreasing or too long");
    }
    for (int s = 0; s < S; ++s) {
        if (b->n_layers[s] < 0 || b->n_layers[s] > NR_MAX_LAYERS) return err(NR_EINVAL, "n_layers out of range");
        if (b->dataset[s] < 0 || b->dataset[s] >= b->n_datasets) return err(NR_EINVAL, "dataset out of range");
    }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The work list is staged in static host arrays that the next call
    // overwrites: a captured copy would replay whatever the latest eager call
    // left there, against the grids fixed at capture time.  So a capturing
    // stream is refused before anything is enqueued.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return err(NR_ECUDA, "cudaStreamIsCapturing failed");
    if (cap != cudaStreamCaptureStatusNone)
        return err(NR_EINVAL, "nr_loglik_grad_noalloc cannot be captured in a CUDA graph (its work list is "
                              "staged in host memory that every call rewrites)");

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return err(NR_ECUDA, "cudaGetDevice failed");
    if (!g_scratch_dev[dev]) {
        // one-time set-up on this device (must precede any stream capture)
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return err(NR_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
        g_scratch_dev[dev] = ptr;
    }
    unsigned char *base = static_cast<unsigned char *>(g_scratch_dev[dev]);
    int32_t *d_tickets = reinterpret_cast<int32_t *>(base);
    int32_t *d_status = d_tickets + 2 * kNumBuckets;
    StackInfo *d_stacks = reinterpret_cast<StackInfo *>(base + kCtrlBytes);
    WorkItem *d_items = reinterpret_cast<WorkItem *>(base + kCtrlBytes + (size_t)kMaxStacks * sizeof(StackInfo));

    // one work item per stack; items grouped by bucket, longest first
    int64_t par = 0, out = 0;
    int count[kNumBuckets] = {};
    for (int s = 0; s < S; ++s) {
        StackInfo &si = h_stacks[s];
        const int n = b->n_layers[s];
        const int64_t q0 = b->q_off[b->dataset[s]];
        si.par_off = par;
        si.out_off = out;
        si.q_begin = q0;
        si.part_base = 0;
        si.n = n;
        si.nq = (int32_t)(b->q_off[b->dataset[s] + 1] - q0);
        si.n_chunks = 1;
        si.pad = 0;
        par += 4 * (int64_t)n + 6;
        out += si.nq;
        h_order[s] = s;
        count[bucket_of(n)]++;
    }
    std::sort(h_order, h_order + S, [&](int x, int y) {
        const int bx = bucket_of(h_stacks[x].n), by = bucket_of(h_stacks[y].n);
        if (bx != by) return bx < by;
        const int64_t cx = (int64_t)(h_stacks[x].n + 1) * h_stacks[x].nq, cy = (int64_t)(h_stacks[y].n + 1) * h_stacks[y].nq;
        if (cx != cy) return cx > cy;
        return x < y;
    });
    for (int i = 0; i < S; ++i) {
        const int s = h_order[i];
        h_items[i].stack = s;
        h_items[i].q_lo = 0;
        h_items[i].q_hi = h_stacks[s].nq;
        h_items[i].chunk = 0;
    }

    // what must start at zero: queue tickets and status word
    if (cudaMemsetAsync(base, 0, kCtrlBytes, st) != cudaSuccess) return err(NR_ECUDA, "cudaMemsetAsync failed");
    if (device_flags && cudaMemsetAsync(device_flags, 0, sizeof(int32_t), st) != cudaSuccess)
        return err(NR_ECUDA, "cudaMemsetAsync failed");
    if (cudaMemcpyAsync(d_stacks, h_stacks, sizeof(StackInfo) * S, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_items, h_items, sizeof(WorkItem) * S, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return err(NR_ECUDA, "cudaMemcpyAsync of the work list failed");

    QuadConst qc{};
    if (!make_quad_const(n_quad, qc)) return err(NR_EINVAL, "quadrature failed");
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return err(NR_ECUDA, "cudaDeviceGetAttribute failed");

    KernelArgs a{};
    a.params = b->params;
    a.q = b->q;
    a.dq = b->dq;
    a.r_obs = b->r_obs;
    a.r_err = b->r_err;
    a.stacks = d_stacks;
    a.ll_out = loglik;
    a.grad_out = grad;
    a.status = device_flags ? device_flags : d_status;
    a.n_stacks = S;
    int first = 0;
    for (int g = 0; g < kNumBuckets; ++g) {
        if (count[g] == 0) continue;
        const int nmax = kBuckets[g];
        int occ = 1;
        if (mixed_occupancy(kGrad, nmax, n_quad, &occ) != cudaSuccess) return err(NR_ECUDA, "occupancy query failed");
        a.items = d_items + first;
        a.n_items = count[g];
        a.tile_q = std::max(1, mixed_tile_q(kGrad, nmax, n_quad));
        a.ticket = d_tickets + 2 * g;
        const int grid = std::max(1, std::min(count[g], sms * std::max(occ, 1)));
        if (launch_mixed(kGrad, nmax, grid, a, qc, st) != cudaSuccess) return err(NR_ECUDA, "kernel launch failed");
        first += count[g];
    }
    return NR_OK;
}
