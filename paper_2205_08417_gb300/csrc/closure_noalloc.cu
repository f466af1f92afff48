// Allocation-free variant of the entropy closure (kitrt_closure_noalloc).
//
// Some callers cannot let the library allocate device memory when they call it: code that runs
// while its framework's pool allocator owns all free device memory (a cudaMalloc there fails or
// makes the pool give memory back), or a long-running service that must not grow its footprint
// after start-up. kitrt_closure needs the solver's mesh-sized workspace; this entry point instead
// solves the closure of any batch of up to a fixed number of moment vectors with its Newton
// scratch in one file-scope device array, so a call allocates nothing.
//
// The scratch array is kScratchBytes (8 MiB) per GPU that loads the library and stays resident
// until the process exits. Every call shares it and it keeps the last call's contents; the call
// clears the counters that must start at zero and every per-cell field is written before it is
// read. Calls that overlap on the GPU (two streams, or two host threads) race on the array. The
// host reads the counters back (and synchronises with the stream) once every four sweeps.
#include <mutex>
#include <string.h>

#include "kitrt_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_closure_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of scratch one cell needs at n moments: doubles alpha, dir, U (3n), fsum, f0, gd, lam (4)
// and the packed Cholesky factor (n(n+1)/2); int32 phase, iters, halv, evals, status and two list
// slots (7); the layout pads each array to 256 bytes, which noalloc_layout accounts for.
struct Layout {
    size_t off[16];
    size_t total;
};

Layout noalloc_layout(int n, int C)
{
    const int npairs = n * (n + 1) / 2;
    const size_t sizes[] = {
        8 * sizeof(int32_t),                   // counters
        (size_t)C * n * sizeof(double),        // alpha
        (size_t)C * n * sizeof(double),        // dir
        (size_t)C * n * sizeof(double),        // U
        (size_t)C * sizeof(double),            // fsum
        (size_t)C * sizeof(double),            // f0
        (size_t)C * sizeof(double),            // gd
        (size_t)C * npairs * sizeof(double),   // L
        (size_t)C * sizeof(double),            // lam
        (size_t)C * sizeof(int32_t),           // phase
        (size_t)C * sizeof(int32_t),           // iters
        (size_t)C * sizeof(int32_t),           // halv
        (size_t)C * sizeof(int32_t),           // evals
        (size_t)C * sizeof(int32_t),           // status
        (size_t)C * sizeof(int32_t),           // list 0
        (size_t)C * sizeof(int32_t),           // list 1
    };
    Layout L;
    size_t o = 0;
    for (int i = 0; i < 16; ++i) {
        L.off[i] = o;
        o += align256(sizes[i]);
    }
    L.total = o;
    return L;
}

// Largest batch whose scratch layout fits the array.
int noalloc_max_cells(int n)
{
    int lo = 0, hi = 1 << 24;
    while (lo < hi) {  // largest C whose layout fits
        int mid = lo + (hi - lo + 1) / 2;
        if (noalloc_layout(n, mid).total <= kScratchBytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace

extern "C" int32_t kitrt_closure_noalloc(const kitrt_mn *mn, const double *u, double *alpha,
                                         int32_t *status, int32_t ncells, void *stream)
{
    if (!mn || !u || !alpha || ncells < 0) return KITRT_EINVAL;
    if (ncells == 0) return KITRT_OK;
    if (ncells > noalloc_max_cells(mn->n)) return KITRT_ESCRATCH;
    cudaStream_t s = (cudaStream_t)stream;

    // set-up, once per device, with that device current: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KITRT_ECUDA;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_closure_scratch) != cudaSuccess || !p) return KITRT_ECUDA;
            g_scratch_ptr[dev] = p;
        }
        base = (unsigned char *)g_scratch_ptr[dev];
    }

    const int n = mn->n, C = ncells;
    const Layout L = noalloc_layout(n, C);
    NewtonState S{};
    S.cnt = (int32_t *)(base + L.off[0]);
    S.alpha = (double *)(base + L.off[1]);
    S.dir = (double *)(base + L.off[2]);
    S.U = (double *)(base + L.off[3]);
    S.fsum = (double *)(base + L.off[4]);
    S.f0 = (double *)(base + L.off[5]);
    S.gd = (double *)(base + L.off[6]);
    S.L = (double *)(base + L.off[7]);
    S.lam = (double *)(base + L.off[8]);
    S.phase = (int32_t *)(base + L.off[9]);
    S.iters = (int32_t *)(base + L.off[10]);
    S.halv = (int32_t *)(base + L.off[11]);
    S.evals = (int32_t *)(base + L.off[12]);
    S.status = (int32_t *)(base + L.off[13]);
    S.list[0] = (int32_t *)(base + L.off[14]);
    S.list[1] = (int32_t *)(base + L.off[15]);

    // launch-geometry view of the solver (no workspace, no tracing)
    kitrt_mn view;
    view.N = mn->N;
    view.n = mn->n;
    view.nsm = mn->nsm;
    const Tables T = mn->tables();
    NewtonParams np{mn->p.tau, mn->p.armijo_c1, mn->p.max_iter, mn->p.max_halvings, mn->p.polish,
                    mn->p.reg_gamma, mn->p.reg_keep_mass ? 1 : 0};

    if (cudaMemsetAsync(S.cnt, 0, 8 * sizeof(int32_t), s) != cudaSuccess) return KITRT_ECUDA;
    int rc = launch_begin(&view, T, S, C, u, alpha, 1, np, s);
    if (rc) return rc;
    const int batch = 4;
    const int max_launch = (mn->p.max_iter + 1) * (mn->p.max_halvings + 1) + 1;
    int32_t cnt[8];
    int k = 0;
    for (;;) {
        for (int b = 0; b < batch; ++b, ++k) {
            rc = launch_eval_fp64(&view, T, S, C, u, k, np, s);
            if (rc) return rc;
        }
        if (cudaMemcpyAsync(cnt, S.cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return KITRT_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return KITRT_ECUDA;
        if (cnt[k % 3] == 0) break;
        if (k >= max_launch) return KITRT_ETIMEOUT;
    }
    rc = launch_finish(&view, T, S, C, alpha, nullptr, nullptr, mn->p.polish, 0, s);
    if (rc) return rc;
    if (status && cudaMemcpyAsync(status, S.status, sizeof(int32_t) * C, cudaMemcpyDeviceToDevice,
                                  s) != cudaSuccess)
        return KITRT_ECUDA;
    if (cnt[3] > 0) {
        // first failing code, read back through a small fixed host buffer
        int32_t chunk[256];
        for (int c0 = 0; c0 < C; c0 += 256) {
            const int m = C - c0 < 256 ? C - c0 : 256;
            if (cudaMemcpyAsync(chunk, S.status + c0, sizeof(int32_t) * m, cudaMemcpyDeviceToHost,
                                s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
                return KITRT_ECUDA;
            for (int i = 0; i < m; ++i)
                if (chunk[i]) return chunk[i];
        }
    }
    return KITRT_OK;
}
