// Batched ensembles of independent 2-D domains of uneven sizes, advanced by one
// persistent kernel per lbm_batch_step call, launched from a captured CUDA graph.
//
// Work items are (step, domain, tile) in step-major order; every CTA of the
// persistent grid takes the next item from a global counter.  An item of step s
// of domain d may start once all items of step s-1 of d have finished (a
// per-domain completion counter); the wait is a bounded spin that sets an error
// flag when it gives up, after which every CTA leaves.  Because items are taken
// in step-major order, an item waits only on items already taken by running
// CTAs, so the grid (sized to be fully resident) cannot deadlock.  Populations
// are read through L2 (ld.global.cg) since other CTAs of the same launch wrote
// them.  Each tile runs the same body as the per-step fused kernel.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <vector>

#include "../../include/evlbm.h"
#include "fused2d_tile.cuh"
#include "trace.h"

namespace evlbm {
namespace {

using namespace fused;

struct BatchDomain {
    unsigned long long off;      // first population element of the domain ([Q][ny][nx] block)
    unsigned long long foff;     // first node of the domain in the per-node field arrays
    int nx, ny;
    int strips, chunks, H;
    int items, base;             // tiles per step, prefix sum of tiles over earlier domains
};

struct BatchArgs {
    const float *popA_f, *popA_g;   // state at the start of the launch
    float *popB_f, *popB_g;          // spare buffer
    const float *RT_iso;             // frozen R*T of all domains (thermal = 0)
    const BatchDomain *dom;
    int n_domains, items_per_step, n_steps;
    unsigned *done;                  // per-domain completed items (all steps of the launch)
    unsigned *next;                  // global work counter (n_steps * items_per_step < 2^31)
    int *error;                      // 1: a wait gave up
    const int *probe;                // test hook: a flag nothing sets (NULL = off)
    long long wait_limit;            // polls before a wait gives up
    int eos;
    float a, b, kappa, lambda, c_eq, c_star;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_i(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int kW, bool THERMAL>
__global__ void __launch_bounds__(threads_of<kW>(), Shape<kW>::MINB) k_batch(BatchArgs B)
{
    extern __shared__ v2 smem[];
    __shared__ int s_item, s_dom, s_ok;
    // The host splits a call so that one launch hands out fewer than 2^31 items.
    const int total = B.n_steps * B.items_per_step;
    for (;;) {
        if (threadIdx.x == 0) {
            int item = -1, d = 0, ok = 0;
            if (!ld_acquire_i(B.error)) {
                const unsigned g = atomicAdd(B.next, 1u);
                if (g < (unsigned)total) {
                    item = (int)g;
                    const int step = item / B.items_per_step, r = item % B.items_per_step;
                    int lo = 0, hi = B.n_domains - 1;          // last domain with base <= r
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) / 2;
                        if (B.dom[mid].base <= r) lo = mid;
                        else hi = mid - 1;
                    }
                    d = lo;
                    ok = 1;
                    const unsigned need = (unsigned)step * (unsigned)B.dom[d].items;
                    long long polls = 0;
                    while (ok && ld_acquire(B.done + d) < need) {
                        if (++polls > B.wait_limit || ld_acquire_i(B.error)) ok = 0;
                        else __nanosleep(64);
                    }
                    if (ok && B.probe) {
                        polls = 0;
                        while (ok && ld_acquire_i(B.probe) == 0) {
                            if (++polls > B.wait_limit) ok = 0;
                            else __nanosleep(64);
                        }
                    }
                    if (!ok) atomicExch(B.error, 1);
                }
            }
            s_item = item;
            s_dom = d;
            s_ok = ok;
        }
        __syncthreads();
        const int item = s_item, d = s_dom, ok = s_ok;
        __syncthreads();
        if (!ok) break;
        const int step = item / B.items_per_step;
        const BatchDomain D = B.dom[d];
        const int k = item % B.items_per_step - D.base;
        FusedArgs A;
        const bool odd = step & 1;
        A.f = (odd ? B.popB_f : B.popA_f) + D.off;
        A.g = THERMAL ? (odd ? B.popB_g : B.popA_g) + D.off : nullptr;
        A.fo = (odd ? const_cast<float *>(B.popA_f) : B.popB_f) + D.off;
        A.go = THERMAL ? (odd ? const_cast<float *>(B.popA_g) : B.popB_g) + D.off : nullptr;
        A.RT_iso = THERMAL ? nullptr : B.RT_iso + D.foff;
        A.Rin = nullptr;
        A.Rout = nullptr;
        A.nx = D.nx;
        A.ny = D.ny;
        A.nz = 1;
        A.H = D.H;
        A.N = (unsigned)D.nx * (unsigned)D.ny;
        A.eos = B.eos;
        A.a = B.a;
        A.b = B.b;
        A.kappa = B.kappa;
        A.lambda = B.lambda;
        A.c_eq = B.c_eq;
        A.c_star = B.c_star;
        A.walls = 0;
        A.wall_uy[0] = A.wall_uy[1] = A.wall_RT = 0.f;
        const int y0 = (k / D.strips) * D.H;
        fused_tile<kW, THERMAL, true>(A, k % D.strips, y0, min(D.H, D.ny - y0), 0, smem);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(B.done + d, 1u);
        }
    }
}

template <int W, bool THERMAL>
cudaError_t launch_batch_w(const BatchArgs &B, int grid, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_batch<W, THERMAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_of<W>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_batch<W, THERMAL><<<grid, threads_of<W>(), smem_of<W>(), st>>>(B);
    return cudaGetLastError();
}

template <int W, bool THERMAL>
int resident_grid()
{
    cudaFuncSetAttribute(k_batch<W, THERMAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of<W>());
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<W, THERMAL>, threads_of<W>(),
                                                      smem_of<W>()) != cudaSuccess)
        return 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

template <bool THERMAL>
cudaError_t launch_batch(int W, const BatchArgs &B, int grid, cudaStream_t st)
{
    switch (W) {
    case 64: return launch_batch_w<64, THERMAL>(B, grid, st);
    case 96: return launch_batch_w<96, THERMAL>(B, grid, st);
    case 192: return launch_batch_w<192, THERMAL>(B, grid, st);
    default: return launch_batch_w<128, THERMAL>(B, grid, st);
    }
}

template <bool THERMAL>
int grid_for(int W)
{
    switch (W) {
    case 64: return resident_grid<64, THERMAL>();
    case 96: return resident_grid<96, THERMAL>();
    case 192: return resident_grid<192, THERMAL>();
    default: return resident_grid<128, THERMAL>();
    }
}

}  // namespace

EVLBM_DEFINE_OOB_READER(batch_oob)

}  // namespace evlbm

using evlbm::BatchArgs;
using evlbm::BatchDomain;
using evlbm::KParams;

struct lbm_batch {
    lbm_params P;
    int n;
    std::vector<int> nx, ny;
    std::vector<BatchDomain> dom;
    long long nodes;
    cudaStream_t stream;
    bool own_stream;             // created here because the caller passed NULL
    float *f[2], *g[2];
    float *RT_iso;
    int cur;
    BatchDomain *d_dom;
    unsigned *d_done, *d_next;
    int *d_error, *d_probe;
    int tile_w, tile_h;
    long long wait_limit;
    bool probe_on;
    int items_per_step;
    cudaGraphExec_t graph;
    int graph_steps, graph_cur, graph_w, graph_h;
    bool graph_probe;
    long long graph_limit;
    void *scratch;               // stage-kernel fields for lbm_batch_moments (largest domain)
    long long max_nodes;
    long long steps;
    KParams K;                   // common physics (per-domain sizes filled on use)
    char err[512];
};

namespace {

int bfail(lbm_batch *b, int code, const char *fmt, ...)
{
    static thread_local char init_err[512];
    char *dst = b ? b->err : init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return code;
}

#define BCK(b, call)                                                                              \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", #call, \
                         cudaGetErrorString(e_));                                                 \
    } while (0)

// Recomputes the tiling of every domain for the current launch shape and uploads it.
int retile(lbm_batch *b)
{
    int base = 0;
    const int W = b->tile_w;
    for (int d = 0; d < b->n; ++d) {
        BatchDomain &D = b->dom[d];
        // Equal chunks of at most tile_h rows (even), so that no domain ends in a
        // short chunk that pays the pipeline fill for a few rows.
        const int Hmax = b->tile_h < D.ny ? b->tile_h : D.ny;
        int H = (D.ny + (D.ny + Hmax - 1) / Hmax - 1) / ((D.ny + Hmax - 1) / Hmax);
        H += H & 1;
        D.H = H;
        D.strips = (D.nx + W - 1) / W;
        D.chunks = (D.ny + H - 1) / H;
        D.items = D.strips * D.chunks;
        D.base = base;
        base += D.items;
    }
    b->items_per_step = base;
    BCK(b, cudaMemcpyAsync(b->d_dom, b->dom.data(), sizeof(BatchDomain) * b->n, cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

BatchArgs make_args(const lbm_batch *b, int n_steps)
{
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    const int c = b->cur;
    B.popA_f = b->f[c];
    B.popA_g = b->g[c];
    B.popB_f = b->f[c ^ 1];
    B.popB_g = b->g[c ^ 1];
    B.RT_iso = b->RT_iso;
    B.dom = b->d_dom;
    B.n_domains = b->n;
    B.items_per_step = b->items_per_step;
    B.n_steps = n_steps;
    B.done = b->d_done;
    B.next = b->d_next;
    B.error = b->d_error;
    B.probe = b->probe_on ? b->d_probe : nullptr;
    B.wait_limit = b->wait_limit;
    B.eos = b->P.eos;
    B.a = float(b->P.a);
    B.b = float(b->P.b);
    B.kappa = float(b->P.kappa);
    B.lambda = float(b->P.lambda);
    B.c_eq = float(b->K.c_eq);
    B.c_star = float(b->K.c_star);
    return B;
}

cudaError_t enqueue(lbm_batch *b, int n_steps)
{
    cudaError_t e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned) * b->n, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_error, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    const BatchArgs B = make_args(b, n_steps);
    const int grid = b->P.thermal ? evlbm::grid_for<true>(b->tile_w) : evlbm::grid_for<false>(b->tile_w);
    if (grid <= 0) return cudaErrorLaunchOutOfResources;
    return b->P.thermal ? evlbm::launch_batch<true>(b->tile_w, B, grid, b->stream)
                        : evlbm::launch_batch<false>(b->tile_w, B, grid, b->stream);
}

void drop_graph(lbm_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = -1;
}

// Runs n_steps as one persistent launch from a captured graph; the graph is
// re-captured when the step count, buffer parity, shape or test hooks change.
int run_graph(lbm_batch *b, int n_steps)
{
    if (!b->graph || b->graph_steps != n_steps || b->graph_cur != b->cur || b->graph_w != b->tile_w ||
        b->graph_h != b->tile_h || b->graph_probe != b->probe_on || b->graph_limit != b->wait_limit) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const cudaError_t e = enqueue(b, n_steps);
        const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(b, LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        const cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) return bfail(b, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e3));
        b->graph_steps = n_steps;
        b->graph_cur = b->cur;
        b->graph_w = b->tile_w;
        b->graph_h = b->tile_h;
        b->graph_probe = b->probe_on;
        b->graph_limit = b->wait_limit;
    }
    BCK(b, cudaGraphLaunch(b->graph, b->stream));
    int err = 0;
    BCK(b, cudaMemcpyAsync(&err, b->d_error, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (err) return bfail(b, LBM_ETIMEOUT, "a per-domain step wait gave up (limit %lld polls)", b->wait_limit);
    return LBM_OK;
}

void free_batch(lbm_batch *b)
{
    drop_graph(b);
    for (int k = 0; k < 2; ++k) {
        if (b->f[k]) cudaFree(b->f[k]);
        if (b->g[k]) cudaFree(b->g[k]);
    }
    if (b->RT_iso) cudaFree(b->RT_iso);
    if (b->d_dom) cudaFree(b->d_dom);
    if (b->d_done) cudaFree(b->d_done);
    if (b->d_next) cudaFree(b->d_next);
    if (b->d_error) cudaFree(b->d_error);
    if (b->d_probe) cudaFree(b->d_probe);
    if (b->scratch) cudaFree(b->scratch);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    b->stream = nullptr;
}

}  // namespace

// Steps one persistent launch may take: its work counter hands out n_steps x
// items_per_step items as 32-bit values (kept below 2^31); an even count keeps the
// buffer parity, so the captured graph of a long call is reused for every launch.
extern "C" int lbm_batch_launch_steps(int items_per_step)
{
    if (items_per_step < 1) return -1;
    const long long per = ((1LL << 31) - 1) / items_per_step;
    return per >= 2 ? (int)(per & ~1LL) : 1;
}

namespace {

int batch_launch_steps(int items_per_step) { return lbm_batch_launch_steps(items_per_step); }

KParams domain_kparams(const lbm_batch *b, int d)
{
    KParams k = b->K;
    k.nx = b->dom[d].nx;
    k.ny = b->dom[d].ny;
    k.nz = 1;
    k.N = (long long)k.nx * k.ny;
    return k;
}

}  // namespace

extern "C" {

int lbm_batch_init(const lbm_params *p, int n_domains, const int *nx, const int *ny, const double *rho,
                   const double *u, const double *T, void *stream, lbm_batch **out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!p || n_domains < 1 || !nx || !ny || !rho || !u || !T) return LBM_EINVAL;
    if (p->lattice != LBM_D2Q9 || p->precision != LBM_FP32 || p->force_form != 0 || p->nz != 1)
        return LBM_EINVAL;
    if (!(p->tau > 0.0) || !(p->lambda > 0.0) || !(p->R > 0.0) || !(p->a >= 0.0) || !(p->b >= 0.0) ||
        !(p->kappa >= 0.0) || (p->thermal != 0 && p->thermal != 1) || (p->eos != 0 && p->eos != 1))
        return LBM_EINVAL;
    long long nodes = 0, max_nodes = 0;
    for (int d = 0; d < n_domains; ++d) {
        if (nx[d] < 1 || ny[d] < 1) return LBM_EINVAL;
        const long long Nd = (long long)nx[d] * ny[d];
        if (9 * Nd >= (1LL << 31)) return LBM_EINVAL;
        nodes += Nd;
        max_nodes = Nd > max_nodes ? Nd : max_nodes;
    }
    for (long long k = 0; k < nodes; ++k)
        if (!(rho[k] > 0.0) || !(T[k] > 0.0)) return LBM_ENONFINITE;

    lbm_batch *b = new lbm_batch();
    b->P = *p;
    b->n = n_domains;
    b->nx.assign(nx, nx + n_domains);
    b->ny.assign(ny, ny + n_domains);
    b->dom.resize(n_domains);
    b->nodes = nodes;
    b->max_nodes = max_nodes;
    b->stream = static_cast<cudaStream_t>(stream);
    if (!b->stream) {
        // The legacy default stream cannot be captured into a graph.
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return LBM_ECUDA;
        }
        b->own_stream = true;
    }
    b->tile_w = 128;
    b->tile_h = 128;
    b->wait_limit = 1LL << 24;
    b->graph_steps = -1;
    memset(&b->K, 0, sizeof(KParams));
    b->K.eos = p->eos;
    b->K.thermal = p->thermal;
    b->K.force_form = 0;
    b->K.a = p->a;
    b->K.b = p->b;
    b->K.kappa = p->kappa;
    b->K.lambda = p->lambda;
    const double beta = 1.0 / (2.0 * p->tau + 1.0);     // Eq. (beta), dt = 1
    b->K.c_eq = 2.0 * beta;
    b->K.c_star = (1.0 / p->lambda) * (1.0 - beta);
    unsigned long long off = 0, foff = 0;
    for (int d = 0; d < n_domains; ++d) {
        b->dom[d].off = off;
        b->dom[d].foff = foff;
        b->dom[d].nx = nx[d];
        b->dom[d].ny = ny[d];
        off += 9ULL * nx[d] * ny[d];
        foff += (unsigned long long)nx[d] * ny[d];
    }
    const size_t pop = sizeof(float) * off;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaMalloc(&b->f[k], pop);
        if (e == cudaSuccess && p->thermal) e = cudaMalloc(&b->g[k], pop);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->RT_iso, sizeof(float) * nodes);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_dom, sizeof(BatchDomain) * n_domains);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_done, sizeof(unsigned) * n_domains);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_probe, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_probe, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->scratch, sizeof(float) * evlbm::kRefFieldCount * max_nodes);
    float *d_fields = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_fields, sizeof(float) * 4 * max_nodes);
    if (e != cudaSuccess) {
        const int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
        if (d_fields) cudaFree(d_fields);
        free_batch(b);
        delete b;
        return code;
    }
    // Initial equilibria per domain (host fields are concatenated in domain order;
    // u of a domain is [2][N_d]).
    std::vector<float> h(4 * max_nodes), rt(nodes);
    const double *ud = u;
    for (int d = 0; d < n_domains && e == cudaSuccess; ++d) {
        const long long Nd = (long long)nx[d] * ny[d], f0 = (long long)b->dom[d].foff;
        for (long long k = 0; k < Nd; ++k) {
            h[k] = float(rho[f0 + k]);
            h[Nd + k] = float(ud[k]);
            h[2 * Nd + k] = float(ud[Nd + k]);
            h[3 * Nd + k] = float(p->R * T[f0 + k]);
            rt[f0 + k] = h[3 * Nd + k];
        }
        ud += 2 * Nd;
        e = cudaMemcpyAsync(d_fields, h.data(), sizeof(float) * 4 * Nd, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        const KParams K = domain_kparams(b, d);
        if (e == cudaSuccess)
            e = evlbm::ref_init_f32(1, 9, K, d_fields, d_fields + Nd, d_fields + 3 * Nd, b->f[0] + b->dom[d].off,
                                    p->thermal ? b->g[0] + b->dom[d].off : nullptr, nullptr, b->stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->RT_iso, rt.data(), sizeof(float) * nodes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d_fields);
    if (e != cudaSuccess) {
        free_batch(b);
        delete b;
        return LBM_ECUDA;
    }
    int rc = retile(b);
    if (rc) {
        free_batch(b);
        delete b;
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch *b, int n_steps)
{
    evtrace::Range trace_("lbm_batch_step");
    if (!b || n_steps < 0) return LBM_EINVAL;
    int left = n_steps;
    while (left > 0) {
        const int n = left < batch_launch_steps(b->items_per_step) ? left : batch_launch_steps(b->items_per_step);
        const int rc = run_graph(b, n);
        if (rc) return rc;
        b->cur ^= (n & 1);
        b->steps += n;
        left -= n;
    }
    return LBM_OK;
}

int lbm_batch_set_tile(lbm_batch *b, int tile_w, int tile_h)
{
    if (!b) return LBM_EINVAL;
    bool ok = false;
    for (int k = 0; k < evlbm::kFusedWidthCount; ++k) ok = ok || tile_w == evlbm::kFusedWidths[k];
    if (!ok || tile_h < 1) return bfail(b, LBM_EINVAL, "tile_w must be one of 64,96,128,192 and tile_h >= 1");
    b->tile_w = tile_w;
    b->tile_h = tile_h;
    return retile(b);
}

int lbm_batch_get_tile(const lbm_batch *b, int *tile_w, int *tile_h)
{
    if (!b) return LBM_EINVAL;
    if (tile_w) *tile_w = b->tile_w;
    if (tile_h) *tile_h = b->tile_h;
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch *b, int probe_steps, int *tile_w, int *tile_h)
{
    if (!b || probe_steps < 1) return LBM_EINVAL;
    const int heights[] = {32, 64, 128, 256, 512};     // 512: every domain of <= 512 rows in one chunk
    // Each shape is timed on one persistent launch of 2 * probe_steps steps, as in a run,
    // where the last items of a step overlap the first items of the next.  The launch
    // starts from a copy of the current state; an even step count ends in the current
    // buffer, which is restored from the copy before every probe and at the end.  If the
    // copy cannot be allocated, each shape is timed on single-step launches into the spare
    // buffer instead (state untouched).
    const size_t pop = sizeof(float) * 9ULL * (size_t)b->nodes;
    float *save_f = nullptr, *save_g = nullptr;
    bool saved = cudaMalloc(&save_f, pop) == cudaSuccess &&
                 (!b->P.thermal || cudaMalloc(&save_g, pop) == cudaSuccess);
    if (!saved) {
        cudaGetLastError();                   // clear the failed allocation
        if (save_f) cudaFree(save_f);
        save_f = nullptr;
    }
    auto copy_state = [&](bool restore) -> cudaError_t {
        const int c = b->cur;
        cudaError_t e = cudaMemcpyAsync(restore ? b->f[c] : save_f, restore ? save_f : b->f[c], pop,
                                        cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess && b->P.thermal)
            e = cudaMemcpyAsync(restore ? b->g[c] : save_g, restore ? save_g : b->g[c], pop,
                                cudaMemcpyDeviceToDevice, b->stream);
        return e;
    };
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int bw = b->tile_w, bh = b->tile_h;
    int rc = LBM_OK;
    const bool have_copy = saved && copy_state(false) == cudaSuccess;
    if (saved && !have_copy) rc = LBM_ECUDA;
    for (int wi = 0; wi < evlbm::kFusedWidthCount && rc == LBM_OK; ++wi) {
        for (int hi = 0; hi < 5 && rc == LBM_OK; ++hi) {
            b->tile_w = evlbm::kFusedWidths[wi];
            b->tile_h = heights[hi];
            if ((rc = retile(b))) break;
            float ms = 0.f;
            if (saved) {
                if (copy_state(true) != cudaSuccess || cudaEventRecord(e0, b->stream) != cudaSuccess ||
                    enqueue(b, 2 * probe_steps) != cudaSuccess)
                    rc = LBM_ECUDA;
            } else {
                // Single steps from the current state into the spare buffer (no parity change).
                for (int s = 0; s <= probe_steps && rc == LBM_OK; ++s) {
                    if (s == 1 && cudaEventRecord(e0, b->stream) != cudaSuccess) rc = LBM_ECUDA;
                    if (rc == LBM_OK && enqueue(b, 1) != cudaSuccess) rc = LBM_ECUDA;
                }
            }
            if (rc == LBM_OK && cudaEventRecord(e1, b->stream) != cudaSuccess) rc = LBM_ECUDA;
            if (rc == LBM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = LBM_ECUDA;
            if (rc == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = LBM_ECUDA;
            int err = 0;
            if (rc == LBM_OK && cudaMemcpy(&err, b->d_error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = LBM_ECUDA;
            if (rc == LBM_OK && err) rc = LBM_ETIMEOUT;
            if (rc == LBM_OK && ms < best) {
                best = ms;
                bw = b->tile_w;
                bh = b->tile_h;
            }
        }
    }
    if (saved) {
        if (have_copy && (copy_state(true) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess))
            if (rc == LBM_OK) rc = LBM_ECUDA;
        cudaFree(save_f);
        if (save_g) cudaFree(save_g);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tile_w = bw;
    b->tile_h = bh;
    const int rc2 = retile(b);
    if (rc) return bfail(b, rc, "lbm_batch_autotune failed");
    if (rc2) return rc2;
    if (tile_w) *tile_w = bw;
    if (tile_h) *tile_h = bh;
    return LBM_OK;
}

int lbm_batch_set_wait_limit(lbm_batch *b, long long polls, int probe_unset_flag)
{
    if (!b || polls < 1 || (probe_unset_flag != 0 && probe_unset_flag != 1)) return LBM_EINVAL;
    b->wait_limit = polls;
    b->probe_on = probe_unset_flag != 0;
    return LBM_OK;
}

int lbm_batch_moments(lbm_batch *b, int domain, double *rho, double *u, double *T)
{
    if (!b || domain < 0 || domain >= b->n) return LBM_EINVAL;
    const KParams K = domain_kparams(b, domain);
    const BatchDomain &D = b->dom[domain];
    const long long Nd = K.N;
    cudaError_t e = evlbm::ref_macro_f32(1, 9, K, b->scratch, b->RT_iso + D.foff, b->f[b->cur] + D.off,
                                         b->P.thermal ? b->g[b->cur] + D.off : nullptr, nullptr, b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_moments: %s", cudaGetErrorString(e));
    std::vector<float> h(4 * Nd);
    using O = evlbm::FieldOffsets;
    const float *s = static_cast<const float *>(b->scratch);
    BCK(b, cudaMemcpyAsync(h.data(), s + O::rho * Nd, sizeof(float) * Nd, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(h.data() + Nd, s + O::u * Nd, sizeof(float) * 2 * Nd, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(h.data() + 3 * Nd, s + O::RT * Nd, sizeof(float) * Nd, cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    for (long long k = 0; k < Nd; ++k) {
        if (rho) rho[k] = h[k];
        if (u) {
            u[k] = h[Nd + k];
            u[Nd + k] = h[2 * Nd + k];
        }
        if (T) T[k] = double(h[3 * Nd + k]) / b->P.R;
    }
    return LBM_OK;
}

long long lbm_batch_nodes(const lbm_batch *b) { return b ? b->nodes : -1; }

int lbm_batch_free(lbm_batch *b)
{
    if (!b) return LBM_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return LBM_OK;
}

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err : ""; }

}  // extern "C"
