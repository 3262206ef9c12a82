// One FP64 time step with no allocation at all: the stage kernels' scratch
// fields live in a fixed-size array in the library's own device memory.
//
// Some callers cannot allocate device memory while they run: an application
// that hands the GPU to this library from inside a region where cudaMalloc is
// forbidden (a host callback, a pre-planned memory arena whose budget is fixed
// at start-up, or a process whose allocator is owned by another framework)
// still has its populations in device buffers it owns.  lbm_step_noalloc
// serves them: it takes those buffers, allocates nothing, and keeps the
// intermediate fields in kNoallocMaxNodes-sized static storage.
//
// Compiled with --fmad=false like the other FP64 stage kernels, so its
// populations are bit-identical to lbm_step on an FP64 context.
#include <string.h>

#include <atomic>

#include "../../include/evlbm.h"
#include "ref_launch.cuh"

namespace {

// Largest lattice (nodes) the static scratch holds: 31 FP64 fields per node,
// 32768 nodes -> 7.75 MiB of device memory per GPU that loads the library.
constexpr long long kNoallocMaxNodes = 32768;

static __device__ __align__(256) double g_noalloc_scratch[evlbm::kRefFieldCount * kNoallocMaxNodes];

constexpr int kMaxDevices = 64;
// Device address of g_noalloc_scratch per device, looked up once.  Atomic because two
// threads may make their first call on a device at the same time (both store the same
// address).  A device reset unloads the module, so the address is not valid afterwards.
std::atomic<void *> g_scratch_addr[kMaxDevices];

}  // namespace

extern "C" int lbm_step_noalloc(const lbm_params *p, const double *d_f, const double *d_g, const double *d_RT,
                                double *d_f_out, double *d_g_out, void *stream)
{
    if (!p || !d_f || !d_f_out) return LBM_EINVAL;
    if (p->precision != LBM_FP64) return LBM_EINVAL;
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q27) return LBM_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LBM_EINVAL;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N > kNoallocMaxNodes) return LBM_EINVAL;
    if (!(p->tau > 0.0) || !(p->lambda > 0.0) || !(p->R > 0.0) || !(p->a >= 0.0) || !(p->b >= 0.0) ||
        !(p->kappa >= 0.0))
        return LBM_EINVAL;
    if ((p->eos != LBM_EOS_VDW && p->eos != LBM_EOS_CS) || (p->thermal != 0 && p->thermal != 1) ||
        (p->force_form != 0 && p->force_form != 1))
        return LBM_EINVAL;
    if (p->thermal ? (!d_g || !d_g_out) : !d_RT) return LBM_EINVAL;

    // Set-up, once per device with that device current: the host-side name of a
    // __device__ array is not a device address, so ask the runtime for it.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
    void *scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch) return LBM_ECUDA;
        g_scratch_addr[dev].store(scratch, std::memory_order_release);
    }

    evlbm::KParams k;
    memset(&k, 0, sizeof(k));
    k.nx = p->nx;
    k.ny = p->ny;
    k.nz = p->nz;
    k.N = N;
    k.eos = p->eos;
    k.thermal = p->thermal;
    k.force_form = p->force_form;
    k.a = p->a;
    k.b = p->b;
    k.kappa = p->kappa;
    k.lambda = p->lambda;
    const double beta = 1.0 / (2.0 * p->tau + 1.0);   // Eq. (beta), dt = 1
    k.c_eq = 2.0 * beta;
    k.c_star = (1.0 / p->lambda) * (1.0 - beta);
    // Every scratch field is written by an earlier stage of the same step before
    // it is read, so the stale contents of the previous call need no clearing.
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = p->lattice == LBM_D2Q9
                        ? evlbm::ref_step_t<double, double, 9>(k, scratch, d_RT, d_f, d_g, d_f_out,
                                                               d_g_out, nullptr, nullptr, st)
                        : evlbm::ref_step_t<double, double, 27>(k, scratch, d_RT, d_f, d_g, d_f_out,
                                                                d_g_out, nullptr, nullptr, st);
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
