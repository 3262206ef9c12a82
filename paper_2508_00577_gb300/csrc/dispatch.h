// Host-side entry points of the kernel translation units (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include "common.cuh"
#include "dev16.cuh"

namespace evlbm {

// Stage kernels in FP64 (reference order, no contraction): storage FP64.
cudaError_t ref_init_f64(int Q, const KParams &p, const void *rho, const void *u, const void *RT, void *f, void *g,
                         cudaStream_t st);
cudaError_t ref_macro_f64(int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f, const void *g,
                          cudaStream_t st);
cudaError_t ref_step_f64(int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f, const void *g,
                         void *fo, void *go, cudaStream_t st);
cudaError_t ref_export_f64(int Q, const KParams &p, void *scratch, double R, float *rho, float *u, float *T,
                           cudaStream_t st);
cudaError_t expand_f64(int Q, const KParams &p, const void *src, double *dst, int which, cudaStream_t st);

// Stage kernels in FP32; storage 1 = FP32, 2 = FP16, 3 = BF16.  16-bit storage holds
// deviations from each node's own local equilibrium plus that node's reference
// record R ([N] of kRecBytes, dev16.cuh; double-buffered: Rin read, Rout written).
cudaError_t ref_init_f32(int prec, int Q, const KParams &p, const void *rho, const void *u, const void *RT, void *f,
                         void *g, void *Rout, cudaStream_t st);
cudaError_t ref_macro_f32(int prec, int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f,
                          const void *g, const void *Rin, cudaStream_t st);
cudaError_t ref_step_f32(int prec, int Q, const KParams &p, void *scratch, const void *RT_iso, const void *f,
                         const void *g, void *fo, void *go, const void *Rin, void *Rout, cudaStream_t st);
cudaError_t ref_export_f32(int Q, const KParams &p, void *scratch, double R, float *rho, float *u, float *T,
                           cudaStream_t st);
cudaError_t expand_f32(int prec, int Q, const KParams &p, const void *src, const void *R, double *dst, int which,
                       cudaStream_t st);

// Scratch layout of the stage kernels: rho, j, Gam, Pi, lap, A, F, u, RT, theta0, P0, gamma0, flux, wq,
// m_in (mass streaming into each wall node).
constexpr int kRefFieldCount = 31;
struct FieldOffsets {
    static constexpr long long rho = 0, j = 1, Gam = 4, Pi = 5, lap = 14, A = 15, F = 16, u = 19, RT = 22,
                               theta0 = 23, P0 = 24, gamma0 = 25, flux = 26, wq = 29, m_in = 30;
};

// Fused single-pass D2Q9 step (FP32 arithmetic); prec 1/2/3 as above.  The
// launch shape is a strip of tile_w columns marching over chunks of tile_h rows
// (KParams::tile_w/tile_h; 0 = default).
constexpr int kFusedWidthCount = 4;
// tile_h of the D2Q9 kernel that selects the balanced persistent grid (LBM_TILE_BALANCED).
constexpr int kTileBalanced = -1;
extern const int kFusedWidths[kFusedWidthCount];
void fused2d_default_tile(const KParams &p, int *W, int *H);
bool fused2d_supported(int prec, int Q, const KParams &p);
// Fused single-pass D3Q27 step (FP32 arithmetic, divergence force form; storage prec
// 1/2/3 as above, 16-bit storage reading Rin and writing Rout); the x-y tile of 256
// columns is fused3d_tile_w(prec) wide (32 x 8 for FP32, 16 x 16 for 16-bit storage),
// tile_h is the z-chunk height (0 = default).
int fused3d_tile_w(int prec);
bool fused3d_supported(int prec, int Q, const KParams &p);
cudaError_t fused3d_step(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                         const void *RT_iso, const void *Rin, void *Rout, cudaStream_t st);
// Fused single-pass D2Q9 step (FP32 arithmetic, divergence force form; storage prec 1/2/3,
// 16-bit storage reading Rin and writing Rout; wall columns with FP32 storage only).
cudaError_t fused2d_step(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                         const void *RT_iso, const void *Rin, void *Rout, cudaStream_t st);
// Its 16-bit storage instantiations (fused2d16.cu).
cudaError_t fused2d_step16(int prec, const KParams &p, const void *f, const void *g, void *fo, void *go,
                           const void *RT_iso, const void *Rin, void *Rout, cudaStream_t st);

// FP64 totals of the state (mass, momentum x/y/z, energy) and a non-finite flag.
// `work` must hold at least totals_work_bytes(N) bytes.
size_t totals_work_bytes(long long N);
cudaError_t totals(int prec, int Q, const KParams &p, const void *f, const void *g, const void *R, void *work,
                   double *h_out, int *h_nonfinite, cudaStream_t st);

// Maxwell construction in FP64 on the GPU.
cudaError_t coexistence(int eos, double a, double b, double RT, double rho_c, double *h_out, int *h_status);
// Spinodal densities (host); returns 1 above the critical temperature.
int spinodal(int eos, double a, double b, double RT, double rho_c, double out[2]);
// 10-90 % width and tension of the planar square-gradient interface (host).
void interface(int eos, double a, double b, double RT, double kappa, double rv, double rl, double *width,
               double *sigma);

// Out-of-range accesses counted by the fused kernels of a bounds-checked build
// (-DEVLBM_BOUNDS_CHECK): the count, -1 when the library was built without the
// checks, -2 on a CUDA error.
long long fused2d_oob();
long long fused2d16_oob();
long long fused3d_oob();
long long batch_oob();

}  // namespace evlbm
