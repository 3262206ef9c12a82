// Tensor-core GEMM and the elementwise kernels of the learned surrogate.
//
// The convolutions are GEMMs on the 5th-generation tensor cores: BF16 operands
// staged in shared memory by cp.async, tcgen05.mma issued by one thread into an
// FP32 accumulator in tensor memory, and an epilogue that reads the accumulator
// with tcgen05.ld and fuses bias, SiLU, the transposed-convolution pixel shuffle
// or the split-K reduction.  The 3x3 convolutions gather their operand straight
// from the NHWC activations (implicit im2col); the weight gradients read the
// activations as MN-major operands, so no activation is transposed in memory.
#include <stdint.h>

#include "surrogate.cuh"

namespace evsur {

namespace {

constexpr int BM = 128, BK = 64;
constexpr long kWaitLimit = 1L << 24;   // mbarrier polls before a CTA gives up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: lbo = byte stride between core
// matrices along K, sbo = byte stride between 8-row (M or N) groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < kWaitLimit && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity));
    return done != 0;
}

// 16-byte cp.async; an invalid chunk is zero-filled without reading memory.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0));
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }

// Device-side operand description (log2 sizes of the power-of-two grids).
struct Op {
    const bf16 *p;
    int kind, ld, c0, rows;
    int lc, lh, lw;   // log2 C, log2 H, log2 W
};

// Child s = 2 di + dj of coarse pixel q (grid 2^lh x 2^lw) on the 2x finer grid.
__device__ __forceinline__ long long fine_pixel(long long q, int s, int lh, int lw)
{
    const int W = 1 << lw, H = 1 << lh;
    const int x = (int)(q & (W - 1)), y = (int)((q >> lw) & (H - 1));
    const long long b = q >> (lw + lh);
    return (((b << (lh + 1)) | (2 * y + (s >> 1))) << (lw + 1)) | (2 * x + (s & 1));
}

// Per-thread loader state of one operand.  Producer thread t (0..127) owns
// ROWS/16 16-byte chunks of every stage:
//   K-major operands (DENSE, CONV3, UPADJ): rows r_i = (t >> 3) + 16 i, K group t & 7;
//     the rows (pixels) are fixed for the whole K loop, so their coordinates are
//     computed once; a stage only changes the tap.
//   MN-major operands (TDENSE, TCONV3, TUP): row group g = t % (ROWS/8) (fixed: one
//     tap and 8 channels), K indices (pixels) k_j = t / (ROWS/8) + (1024/ROWS) j.
template <int ROWS> struct Loader {
    static constexpr int NCH = ROWS / 16;   // chunks per thread per stage
    int x[NCH], yb[NCH];                     // K-major gathers: pixel x and (sample*H + y)
    bool rv[NCH];                            // K-major: row valid
    long long rowoff[NCH];                   // K-major dense: row offset in elements
    int g, c, dy, dx;                        // MN-major: row group, channel, tap offsets
    bool gv;
};

template <int ROWS>
__device__ __forceinline__ void loader_init(const Op &o, Loader<ROWS> &L, long long row0, int t)
{
    if (o.kind <= SUR_OP_UPADJ) {
#pragma unroll
        for (int i = 0; i < Loader<ROWS>::NCH; ++i) {
            const long long q = row0 + (t >> 3) + 16 * i;
            L.rv[i] = q < o.rows;
            L.rowoff[i] = q * o.ld + o.c0;
            L.x[i] = (int)(q & ((1 << o.lw) - 1));
            L.yb[i] = (int)(q >> o.lw);
        }
    } else {
        constexpr int G = ROWS / 8;
        L.g = t % G;
        const long long r0 = row0 + 8 * L.g;
        L.gv = r0 < o.rows;
        L.c = (int)r0;
        L.dy = L.dx = 0;
        if (o.kind != SUR_OP_TDENSE) {
            const int tap = (int)(r0 >> o.lc);
            L.c = (int)(r0 & ((1 << o.lc) - 1));
            L.gv = L.gv && tap < (o.kind == SUR_OP_TCONV3 ? 9 : 4);
            if (o.kind == SUR_OP_TCONV3) {
                L.dy = ((tap * 11) >> 5) - 1;
                L.dx = tap - 3 * (L.dy + 1) - 1;
            } else {
                L.dy = tap >> 1;   // child offsets di, dj
                L.dx = tap & 1;
            }
        }
    }
}

// Pixel at offset (dy, dx) from (x, yb = sample*H + y), periodic on a 2^lh x 2^lw grid.
__device__ __forceinline__ long long shifted(int x, int yb, int dy, int dx, int lh, int lw)
{
    const int hm = (1 << lh) - 1, wm = (1 << lw) - 1;
    const int ys = (yb & ~hm) | ((yb + dy) & hm);
    return ((long long)ys << lw) | ((x + dx) & wm);
}

// Child (di, dj) on the 2x finer grid of coarse pixel (x, yb).
__device__ __forceinline__ long long child(int x, int yb, int di, int dj, int lw)
{
    return ((long long)(2 * yb + di) << (lw + 1)) | (2 * x + dj);
}

// Fill one operand tile of ROWS x 64 (K) for the K block starting at kbase
// (K indices >= kend read zero).
//   K-major tile: core matrix (row group r/8, k group k/8) at ((r/8)*8 + k/8)*128 B,
//                 row r%8 at +16 B (LBO = 128, SBO = 1024).
//   MN-major tile: core matrix (k group k/8, row group g) at ((k/8)*(ROWS/8) + g)*128 B,
//                 k%8 at +16 B (SBO = 128, LBO = ROWS*16).
template <int ROWS>
__device__ __forceinline__ void load_tile(const Op &o, const Loader<ROWS> &L, uint32_t s, long long kbase,
                                          long long kend, int t)
{
    constexpr int NCH = Loader<ROWS>::NCH;
    if (o.kind <= SUR_OP_UPADJ) {
        const int k8 = t & 7;
        const long long k = kbase + k8 * 8;
        bool kval = k < kend;
        int tap = 0, cc = 0;
        if (o.kind != SUR_OP_DENSE) {
            const int q = (int)(k >> 3);
            tap = q >> (o.lc - 3);
            cc = (q & ((1 << (o.lc - 3)) - 1)) << 3;
            kval = kval && tap < (o.kind == SUR_OP_CONV3 ? 9 : 4);
        }
        int dy, dx;
        if (o.kind == SUR_OP_CONV3) {
            dy = ((tap * 11) >> 5) - 1;
            dx = tap - 3 * (dy + 1) - 1;
        } else {
            dy = tap >> 1;
            dx = tap & 1;
        }
        const uint32_t sk = s + (uint32_t)(k8 * 128 + ((t >> 3) & 7) * 16 + ((t >> 6) << 10));
#pragma unroll
        for (int i = 0; i < NCH; ++i) {
            const bool v = kval && L.rv[i];
            const bf16 *src = o.p;
            if (v) {
                if (o.kind == SUR_OP_DENSE) {
                    src = o.p + L.rowoff[i] + k;
                } else {
                    const long long pix = o.kind == SUR_OP_CONV3 ? shifted(L.x[i], L.yb[i], dy, dx, o.lh, o.lw)
                                                                 : child(L.x[i], L.yb[i], dy, dx, o.lw);
                    src = o.p + pix * o.ld + o.c0 + cc;
                }
            }
            // row r = (t >> 3) + 16 i: group r/8 = (t >> 6) + 2 i, r % 8 = (t >> 3) & 7
            cp_async16(sk + (uint32_t)(i * 2048), src, v);
        }
    } else {
        constexpr int G = ROWS / 8;
        constexpr int KSTEP = 128 / G;
        const int hm = (1 << o.lh) - 1;
        (void)hm;
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const int k = t / G + KSTEP * j;
            const long long q = kbase + k;
            const bool v = L.gv && q < kend;
            const bf16 *src = o.p;
            if (v) {
                long long pix = q;
                if (o.kind != SUR_OP_TDENSE) {
                    const int x = (int)(q & ((1 << o.lw) - 1)), yb = (int)(q >> o.lw);
                    pix = o.kind == SUR_OP_TCONV3 ? shifted(x, yb, L.dy, L.dx, o.lh, o.lw)
                                                  : child(x, yb, L.dy, L.dx, o.lw);
                }
                src = o.p + pix * o.ld + o.c0 + L.c;
            }
            cp_async16(s + (uint32_t)(((k >> 3) * G + L.g) * 128 + (k & 7) * 16), src, v);
        }
    }
}

struct KArgs {
    Op a, b;
    long long M, K;
    int N;
    long long kps;   // K per split, multiple of BK
    int epi;
    const float *bias;
    void *out;
    int ldo, co0;
    bf16 *y;
    int ldy, cy0;
    int shuf_cout, shuf_lh, shuf_lw;
    int *status;
};

template <int BN> struct Cfg {
    static constexpr int NS = BN <= 64 ? 4 : 3;
    static constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = NS * STAGE;
    static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
};

__device__ __forceinline__ uint4 pack8(const float *v)
{
    uint4 r;
    uint32_t *w = reinterpret_cast<uint32_t *>(&r);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&h);
    }
    return r;
}

__device__ __forceinline__ void store32_bf16(bf16 *dst, const float *v)
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = pack8(v + 8 * i);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar));
}

// Bounded wait that also gives up as soon as another role raised the abort flag.
__device__ __forceinline__ bool mbar_wait_abortable(uint32_t bar, uint32_t parity, const volatile int *abort_flag)
{
    uint32_t done = 0;
    for (long it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity));
        if (!done && (it & 63) == 63 && *abort_flag) return false;
    }
    return done != 0;
}

// Warp-specialised GEMM CTA: warps 0-3 produce stages (cp.async) and afterwards
// run the epilogue; warp 4 issues the MMAs.
//   full[s]  (128 arrivals): the producers' copies of stage s have landed and are
//            fenced for the async proxy;
//   empty[s] (tcgen05.commit): the MMAs that read stage s have completed;
//   done     (tcgen05.commit): every MMA of the tile has completed.
template <int BN>
__global__ void __launch_bounds__(160, 1) k_gemm(const KArgs g)
{
    using C = Cfg<BN>;
    constexpr int NS = C::NS;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t full[NS], empty[NS], done_bar;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_flag;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const long long kbeg = (long long)blockIdx.z * g.kps;
    long long kend = kbeg + g.kps;
    if (kend > g.K) kend = g.K;
    const int nkb = kend > kbeg ? (int)((kend - kbeg + BK - 1) / BK) : 0;
    const bool a_mn = g.a.kind >= SUR_OP_TDENSE, b_mn = g.b.kind >= SUR_OP_TDENSE;
    volatile int *abort_v = &abort_flag;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(128));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&done_bar)), "r"(1));
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_sh;
    const uint32_t sbase = smem_u32(dsm);

    if (warp < 4) {
        // ---------------- producers ----------------
        Loader<BM> La;
        Loader<BN> Lb;
        loader_init<BM>(g.a, La, m0, t);
        loader_init<BN>(g.b, Lb, n0, t);
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % NS;
            if (kb >= NS && !mbar_wait_abortable(smem_u32(&empty[s]), ((kb / NS) - 1) & 1, abort_v)) {
                ok = false;
                *abort_v = 1;
                break;
            }
            const uint32_t sa = sbase + (uint32_t)(s * C::STAGE);
            const long long kbase = kbeg + (long long)kb * BK;
            load_tile<BM>(g.a, La, sa, kbase, kend, t);
            load_tile<BN>(g.b, Lb, sa + C::A_BYTES, kbase, kend, t);
            // Arrives on full[s] once this thread's copies above have landed.
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])));
        }
        asm volatile("cp.async.wait_all;");
        // ---------------- epilogue ----------------
        const bool fin = mbar_wait(smem_u32(&done_bar), 0);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (!fin) *abort_v = 1;
        __syncwarp();
        // Warp-uniform decision: tcgen05.ld below is a .sync.aligned warp instruction.
        const bool good = __all_sync(0xffffffffu, fin && !*abort_v && nkb > 0);
        if (good) {
            const long long row = m0 + warp * 32 + lane;
            const bool rv = row < g.M;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (!rv) continue;
                const int col = n0 + c0;
                float v[32];
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) v[jj] = __uint_as_float(r[jj]);
                if (g.epi == SUR_EPI_F32_ATOMIC) {
                    float *o = static_cast<float *>(g.out) + row * g.ldo + g.co0 + col;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) atomicAdd(o + jj, v[jj]);
                } else if (g.epi == SUR_EPI_SHUF) {
                    const int sidx = col / g.shuf_cout, c = col - sidx * g.shuf_cout;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) v[jj] += g.bias[c + jj];
                    const long long q = fine_pixel(row, sidx, g.shuf_lh, g.shuf_lw);
                    store32_bf16(g.y + q * g.ldy + g.cy0 + c, v);
                } else {
                    if (g.bias) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) v[jj] += g.bias[col + jj];
                    }
                    if (g.epi == SUR_EPI_F32) {
                        float4 *o =
                            reinterpret_cast<float4 *>(static_cast<float *>(g.out) + row * g.ldo + g.co0 + col);
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj)
                            o[jj] = make_float4(v[4 * jj], v[4 * jj + 1], v[4 * jj + 2], v[4 * jj + 3]);
                    } else {
                        if (g.out) store32_bf16(static_cast<bf16 *>(g.out) + row * g.ldo + g.co0 + col, v);
                        if (g.epi == SUR_EPI_CONV) {
#pragma unroll
                            for (int jj = 0; jj < 32; ++jj) v[jj] = silu(v[jj]);
                            store32_bf16(g.y + row * g.ldy + g.cy0 + col, v);
                        }
                    }
                }
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer (warp 4, one thread) ----------------
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) |
                               ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % NS;
            if (!mbar_wait_abortable(smem_u32(&full[s]), (kb / NS) & 1, abort_v)) {
                *abort_v = 1;
                break;
            }
            // The stage was written through the generic proxy (cp.async) and is read
            // by the tensor core through the async proxy.
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = sbase + (uint32_t)(s * C::STAGE), sb = sa + C::A_BYTES;
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
                const uint64_t da =
                    a_mn ? smem_desc(sa + k * (BM * 32), BM * 16, 128) : smem_desc(sa + k * 256, 128, 1024);
                const uint64_t db =
                    b_mn ? smem_desc(sb + k * (BN * 32), BN * 16, 128) : smem_desc(sb + k * 256, 128, 1024);
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty[s])));
        }
        // Arrives once every MMA issued above has completed (at once if none was issued).
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done_bar)));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (t == 0 && *abort_v) atomicExch(g.status, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
}

template <int BN>
cudaError_t launch_gemm(const KArgs &g, long long mtiles, int splits, cudaStream_t st)
{
    static int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(k_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<BN>::SMEM);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const dim3 grid((unsigned)mtiles, (unsigned)(g.N / BN), (unsigned)splits);
    k_gemm<BN><<<grid, 160, Cfg<BN>::SMEM, st>>>(g);
    return cudaGetLastError();
}

int ilog2(long long v)
{
    int l = 0;
    while (l < 62 && (1LL << l) < v) ++l;
    return (1LL << l) == v ? l : -1;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Validate a public operand and convert it; false if it is malformed.
bool make_op(const sur_operand &s, Op &o)
{
    if (!s.p || !aligned16(s.p) || s.kind < SUR_OP_DENSE || s.kind > SUR_OP_TUP) return false;
    if (s.ld <= 0 || s.ld % 8 || s.c0 < 0 || s.c0 % 8 || s.rows < 0) return false;
    o.p = static_cast<const bf16 *>(s.p);
    o.kind = s.kind;
    o.ld = s.ld;
    o.c0 = s.c0;
    o.rows = s.rows;
    o.lc = o.lh = o.lw = 0;
    if (s.kind == SUR_OP_DENSE || s.kind == SUR_OP_TDENSE) return true;
    o.lc = ilog2(s.C);
    o.lh = ilog2(s.H);
    o.lw = ilog2(s.W);
    return o.lc >= 3 && o.lh >= 0 && o.lw >= 0 && s.c0 + s.C <= s.ld;
}

}  // namespace

int gemm(const sur_gemm_args &a, int *status, cudaStream_t st)
{
    if (!status || a.M < 1 || a.N < 32 || a.N % 32 || a.K < 1 || a.splits < 1) return SUR_EINVAL;
    if (a.splits > 1 && a.epi != SUR_EPI_F32_ATOMIC) return SUR_EINVAL;
    if (a.epi < SUR_EPI_BF16 || a.epi > SUR_EPI_SHUF) return SUR_EINVAL;
    KArgs g;
    if (!make_op(a.a, g.a) || !make_op(a.b, g.b)) return SUR_EINVAL;
    if (a.b.rows < a.N) return SUR_EINVAL;
    // Chunks are 8 elements wide: a dense operand's K tail and a transposed
    // operand's last row group must stay inside the row of ld elements.
    const long long k8 = (a.K + 7) / 8 * 8;
    for (const sur_operand *o : {&a.a, &a.b}) {
        if (o->kind == SUR_OP_DENSE && o->c0 + k8 > o->ld) return SUR_EINVAL;
        if (o->kind == SUR_OP_TDENSE && o->c0 + (o->rows + 7) / 8 * 8 > o->ld) return SUR_EINVAL;
    }
    g.M = a.M;
    g.N = a.N;
    g.K = a.K;
    const long long kb = (a.K + BK - 1) / BK;
    const long long kbps = (kb + a.splits - 1) / a.splits;
    g.kps = kbps * BK;
    const int splits = (int)((kb + kbps - 1) / kbps);
    g.epi = a.epi;
    g.bias = a.bias;
    g.out = a.out;
    g.ldo = a.ldo;
    g.co0 = a.co0;
    g.y = static_cast<bf16 *>(a.y);
    g.ldy = a.ldy;
    g.cy0 = a.cy0;
    g.shuf_cout = a.shuf_cout;
    g.shuf_lh = g.shuf_lw = 0;
    g.status = status;
    const bool f32 = a.epi == SUR_EPI_F32 || a.epi == SUR_EPI_F32_ATOMIC;
    if (a.epi == SUR_EPI_CONV || a.epi == SUR_EPI_SHUF) {
        if (!a.y || !aligned16(a.y) || !a.bias || a.ldy % 8 || a.cy0 % 8 || a.cy0 < 0) return SUR_EINVAL;
    }
    if (a.epi == SUR_EPI_SHUF) {
        g.shuf_lh = ilog2(a.shuf_H);
        g.shuf_lw = ilog2(a.shuf_W);
        if (g.shuf_lh < 0 || g.shuf_lw < 0 || a.shuf_cout < 32 || a.shuf_cout % 32 || a.N != 4 * a.shuf_cout ||
            a.cy0 + a.shuf_cout > a.ldy)
            return SUR_EINVAL;
    } else if (a.epi == SUR_EPI_CONV) {
        if (a.cy0 + a.N > a.ldy) return SUR_EINVAL;
        if (a.out && (!aligned16(a.out) || a.ldo % 8 || a.co0 % 8 || a.co0 < 0 || a.co0 + a.N > a.ldo))
            return SUR_EINVAL;
    } else {
        if (!a.out || !aligned16(a.out) || a.co0 + a.N > a.ldo || a.co0 < 0) return SUR_EINVAL;
        if (!f32 && (a.ldo % 8 || a.co0 % 8)) return SUR_EINVAL;
        if (a.epi == SUR_EPI_F32 && (a.ldo % 4 || a.co0 % 4)) return SUR_EINVAL;
    }
    const long long mtiles = (a.M + BM - 1) / BM;
    if (mtiles > 0x7FFFFFFF) return SUR_EINVAL;
    cudaError_t e;
    if (a.N % 128 == 0) e = launch_gemm<128>(g, mtiles, splits, st);
    else if (a.N % 64 == 0) e = launch_gemm<64>(g, mtiles, splits, st);
    else e = launch_gemm<32>(g, mtiles, splits, st);
    return e == cudaSuccess ? SUR_OK : SUR_ECUDA;
}

// ---------------------------------------------------------------------------
// Elementwise and reduction kernels.
// ---------------------------------------------------------------------------
namespace {

inline int grid_1d(long long n)
{
    long long g = (n + 255) / 256;
    return (int)(g > 8192 ? 8192 : (g < 1 ? 1 : g));
}

#define GRID_STRIDE(e, total)                                                                    \
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)(total); \
         e += (long long)gridDim.x * blockDim.x)

// dZ = dY * silu'(Z), silu'(z) = s (1 + z (1 - s)) with s = 1 / (1 + e^-z); 8 channels per thread.
__global__ void k_silu_bwd(const bf16 *dY, int ldd, const bf16 *Z, long long M, int C, bf16 *dZ)
{
    const int C8 = C >> 3;
    GRID_STRIDE(e, M * C8)
    {
        const long long m = e / C8;
        const int c = (int)(e - m * C8) << 3;
        const uint4 dv = *reinterpret_cast<const uint4 *>(dY + m * ldd + c);
        const uint4 zv = *reinterpret_cast<const uint4 *>(Z + m * C + c);
        const bf16 *dh = reinterpret_cast<const bf16 *>(&dv), *zh = reinterpret_cast<const bf16 *>(&zv);
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float z = __bfloat162float(zh[j]);
            const float s = 1.f / (1.f + __expf(-z));
            o[j] = __bfloat162float(dh[j]) * s * (1.f + z * (1.f - s));
        }
        *reinterpret_cast<uint4 *>(dZ + m * C + c) = pack8(o);
    }
}

// out[c] += sum over rows of X[m*ldx + c], c < C (bias gradients).  Block (32, 8):
// threadIdx.x picks the column inside a 32-wide slab, rows split over y and the grid.
__global__ void k_colsum(const bf16 *X, int ldx, long long M, int C, float *out)
{
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    float acc = 0.f;
    if (c < C)
        for (long long m = (long long)blockIdx.y * 8 + threadIdx.y; m < M; m += (long long)gridDim.y * 8)
            acc += __bfloat162float(X[m * ldx + c]);
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && c < C) {
        float s = 0.f;
        for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
        atomicAdd(out + c, s);
    }
}

// 2x2 average pooling: X (fine grid, ld ldx, C channels) -> Y [coarse][C], coarse grid 2^lh x 2^lw.
__global__ void k_pool2(const bf16 *X, int ldx, long long Mc, int lh, int lw, int C, bf16 *Y)
{
    GRID_STRIDE(e, Mc * C)
    {
        const long long q = e / C;
        const int c = (int)(e - q * C);
        float s = 0.f;
#pragma unroll
        for (int sidx = 0; sidx < 4; ++sidx) s += __bfloat162float(X[fine_pixel(q, sidx, lh, lw) * ldx + c]);
        Y[e] = __float2bfloat16_rn(0.25f * s);
    }
}

// Adjoint of the pooling, accumulated: dX[fine] += dY[coarse] / 4.
__global__ void k_unpool2_acc(const bf16 *dY, long long Mc, int lh, int lw, int C, bf16 *dX, int ldx)
{
    GRID_STRIDE(e, Mc * C)
    {
        const long long q = e / C;
        const int c = (int)(e - q * C);
        const float d = 0.25f * __bfloat162float(dY[e]);
#pragma unroll
        for (int sidx = 0; sidx < 4; ++sidx) {
            bf16 *p = dX + fine_pixel(q, sidx, lh, lw) * ldx + c;
            *p = __float2bfloat16_rn(__bfloat162float(*p) + d);
        }
    }
}

// Input packing: x fields [4][M] FP32 -> X [M][8] BF16, channels 4..7 zero.
__global__ void k_pack_in(const float *x, long long M, const float *norm, bf16 *X)
{
    GRID_STRIDE(m, M)
    {
        float v[8];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (x[c * M + m] - norm[c]) / norm[4 + c];
#pragma unroll
        for (int c = 4; c < 8; ++c) v[c] = 0.f;
        *reinterpret_cast<uint4 *>(X + m * 8) = pack8(v);
    }
}

// 1x1 head (C -> 4) and its use: mode 0 = loss against targets, mode 1 = next state.
//   o[m][k] = bh[k] + sum_c Y[m][c] Wh[k][c]
//   mode 0: r = o - (y - x)/out_scale; loss += r^2 / (4M); dO[m][k] = 2 r / (4M)
//   mode 1: xn[k][m] = x[k][m] + out_scale[k] o[m][k]
template <int C>
__global__ void k_head(const bf16 *Y, long long M, const float *Wh, const float *bh, const float *norm, const float *x,
                       const float *yt, int mode, float *dO, float *loss, float *xn)
{
    __shared__ float w[4 * C + 4];
    __shared__ float red[256];
    for (int i = threadIdx.x; i < 4 * C; i += blockDim.x) w[i] = Wh[i];
    if (threadIdx.x < 4) w[4 * C + threadIdx.x] = bh[threadIdx.x];
    __syncthreads();
    const float inv = 1.f / (4.f * (float)M);
    float acc = 0.f;
    GRID_STRIDE(m, M)
    {
        float o[4] = {w[4 * C], w[4 * C + 1], w[4 * C + 2], w[4 * C + 3]};
#pragma unroll
        for (int c8 = 0; c8 < C; c8 += 8) {
            const uint4 v = *reinterpret_cast<const uint4 *>(Y + m * C + c8);
            const bf16 *h = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float yv = __bfloat162float(h[j]);
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] += yv * w[k * C + c8 + j];
            }
        }
        if (mode == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float r = o[k] - (yt[k * M + m] - x[k * M + m]) / norm[8 + k];
                acc += r * r;
                dO[m * 4 + k] = 2.f * r * inv;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) xn[k * M + m] = x[k * M + m] + norm[8 + k] * o[k];
        }
    }
    if (mode != 0) return;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

// Head backward (C = 32): dY[m][c] = sum_k dO[m][k] Wh[k][c]; dWh[k][c] += sum_m dO[m][k] Y[m][c];
// dbh[k] += sum_m dO[m][k].  One warp per pixel at a time, lane = channel.
__global__ void k_head_bwd(const bf16 *Y, long long M, const float *Wh, const float *dO, bf16 *dY, float *dWh,
                           float *dbh)
{
    __shared__ float red[8][4 * 32 + 4];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = Wh[k * 32 + lane];
    float gw[4] = {0, 0, 0, 0}, gb = 0.f;
    for (long long m = (long long)blockIdx.x * 8 + wi; m < M; m += (long long)gridDim.x * 8) {
        const float4 d = *reinterpret_cast<const float4 *>(dO + m * 4);
        const float yv = __bfloat162float(Y[m * 32 + lane]);
        dY[m * 32 + lane] = __float2bfloat16_rn(d.x * w[0] + d.y * w[1] + d.z * w[2] + d.w * w[3]);
        gw[0] += d.x * yv;
        gw[1] += d.y * yv;
        gw[2] += d.z * yv;
        gw[3] += d.w * yv;
        if (lane < 4) gb += lane == 0 ? d.x : (lane == 1 ? d.y : (lane == 2 ? d.z : d.w));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[wi][k * 32 + lane] = gw[k];
    if (lane < 4) red[wi][128 + lane] = gb;
    __syncthreads();
    if (wi == 0) {
        for (int k = 0; k < 4; ++k) {
            float s = 0.f;
            for (int j = 0; j < 8; ++j) s += red[j][k * 32 + lane];
            atomicAdd(dWh + k * 32 + lane, s);
        }
        if (lane < 4) {
            float s = 0.f;
            for (int j = 0; j < 8; ++j) s += red[j][128 + lane];
            atomicAdd(dbh + lane, s);
        }
    }
}

// Adam with bias correction on FP32 masters (c1 = 1 - b1^t, c2 = 1 - b2^t).
__global__ void k_adam(float *w, const float *gr, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    GRID_STRIDE(i, n)
    {
        const float g = gr[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 operand copies of a 3x3 convolution from its master Wt [Kp][Cout]:
//   Wb [Cout][Kp]   (forward B operand, K = tap*Cin + ci)
//   Wf [Cin][Kpo]   (adjoint B operand, K = tap*Cout + co, taken at the mirrored tap 8 - tap)
__global__ void k_conv_weights(const float *Wt, int Cin, int Cout, int Kp, int Kpo, bf16 *Wb, bf16 *Wf)
{
    GRID_STRIDE(e, (long long)Cout * Kp)
    {
        const int co = (int)(e / Kp), k = (int)(e % Kp);
        Wb[e] = __float2bfloat16_rn(Wt[(long long)k * Cout + co]);
    }
    if (!Wf) return;
    GRID_STRIDE(e, (long long)Cin * Kpo)
    {
        const int ci = (int)(e / Kpo), k = (int)(e % Kpo);
        float v = 0.f;
        if (k < 9 * Cout) {
            const int tap = k / Cout, co = k % Cout;
            v = Wt[(long long)((8 - tap) * Cin + ci) * Cout + co];
        }
        Wf[e] = __float2bfloat16_rn(v);
    }
}

// BF16 copies of a transposed convolution from its master W [4 Cout][Cin]:
//   Wb [4 Cout][Cin] (forward B operand), Wt [Cin][4 Cout] (adjoint B operand).
__global__ void k_up_weights(const float *Wm, int Cin, int Cout, bf16 *Wb, bf16 *Wt)
{
    GRID_STRIDE(e, 4LL * Cout * Cin)
    {
        const int r = (int)(e / Cin), ci = (int)(e % Cin);
        const bf16 v = __float2bfloat16_rn(Wm[e]);
        Wb[e] = v;
        Wt[(long long)ci * 4 * Cout + r] = v;
    }
}

// Per-domain FP64 sums of rho and of the liquid count (rho > rho_mid), plus a
// non-finite flag over all four fields: out[2b], out[2b+1]; nonfinite[0] |= 1.
__global__ void k_indicators(const float *F, long long M, long long Mb, float rho_mid, double *out, int *nonfinite)
{
    __shared__ double s1[256], s2[256];
    const long long b = blockIdx.y;
    double a1 = 0.0, a2 = 0.0;
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Mb; i += (long long)gridDim.x * blockDim.x) {
        const long long n = b * Mb + i;
        const float r = F[n];
        a1 += r;
        a2 += r > rho_mid ? 1.0 : 0.0;
        if (nonfinite)
            for (int c = 0; c < 4; ++c) bad |= !isfinite(F[c * M + n]);
    }
    if (bad) atomicOr(nonfinite, 1);
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            s1[threadIdx.x] += s1[threadIdx.x + s];
            s2[threadIdx.x] += s2[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(out + 2 * b, s1[0]);
        atomicAdd(out + 2 * b + 1, s2[0]);
    }
}

}  // namespace

cudaError_t silu_bwd(const bf16 *dY, int ldd, const bf16 *Z, long long M, int C, bf16 *dZ, cudaStream_t st)
{
    k_silu_bwd<<<grid_1d(M * C / 8), 256, 0, st>>>(dY, ldd, Z, M, C, dZ);
    return cudaGetLastError();
}

cudaError_t colsum(const bf16 *X, int ldx, long long M, int C, float *out, cudaStream_t st)
{
    long long gy = (M + 8 * 64 - 1) / (8 * 64);
    if (gy > 1024) gy = 1024;
    const dim3 grid((C + 31) / 32, (unsigned)(gy < 1 ? 1 : gy)), block(32, 8);
    k_colsum<<<grid, block, 0, st>>>(X, ldx, M, C, out);
    return cudaGetLastError();
}

cudaError_t pool2(const bf16 *X, int ldx, long long Mc, int lh, int lw, int C, bf16 *Y, cudaStream_t st)
{
    k_pool2<<<grid_1d(Mc * C), 256, 0, st>>>(X, ldx, Mc, lh, lw, C, Y);
    return cudaGetLastError();
}

cudaError_t unpool2_acc(const bf16 *dY, long long Mc, int lh, int lw, int C, bf16 *dX, int ldx, cudaStream_t st)
{
    k_unpool2_acc<<<grid_1d(Mc * C), 256, 0, st>>>(dY, Mc, lh, lw, C, dX, ldx);
    return cudaGetLastError();
}

cudaError_t pack_in(const float *x, long long M, const float *norm, bf16 *X, cudaStream_t st)
{
    k_pack_in<<<grid_1d(M), 256, 0, st>>>(x, M, norm, X);
    return cudaGetLastError();
}

cudaError_t head(const bf16 *Y, long long M, const float *Wh, const float *bh, const float *norm, const float *x,
                 const float *yt, int mode, float *dO, float *loss, float *xn, cudaStream_t st)
{
    k_head<32><<<grid_1d(M), 256, 0, st>>>(Y, M, Wh, bh, norm, x, yt, mode, dO, loss, xn);
    return cudaGetLastError();
}

cudaError_t head_bwd(const bf16 *Y, long long M, const float *Wh, const float *dO, bf16 *dY, float *dWh, float *dbh,
                     cudaStream_t st)
{
    long long g = (M + 8 * 32 - 1) / (8 * 32);
    if (g > 2048) g = 2048;
    k_head_bwd<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(Y, M, Wh, dO, dY, dWh, dbh);
    return cudaGetLastError();
}

cudaError_t adam(float *w, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t st)
{
    k_adam<<<grid_1d(n), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t conv_weights(const float *Wt, int Cin, int Cout, int Kp, int Kpo, bf16 *Wb, bf16 *Wf, cudaStream_t st)
{
    k_conv_weights<<<grid_1d((long long)Cout * Kp), 256, 0, st>>>(Wt, Cin, Cout, Kp, Kpo, Wb, Wf);
    return cudaGetLastError();
}

cudaError_t up_weights(const float *Wm, int Cin, int Cout, bf16 *Wb, bf16 *Wt, cudaStream_t st)
{
    k_up_weights<<<grid_1d(4LL * Cout * Cin), 256, 0, st>>>(Wm, Cin, Cout, Wb, Wt);
    return cudaGetLastError();
}

cudaError_t indicators(const float *F, int batch, long long Mb, float rho_mid, double *out, int *nonfinite,
                       cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 2 * batch, st);
    if (e != cudaSuccess) return e;
    long long gx = (Mb + 255) / 256;
    if (gx > 64) gx = 64;
    const dim3 grid((unsigned)gx, (unsigned)batch);
    k_indicators<<<grid, 256, 0, st>>>(F, (long long)batch * Mb, Mb, rho_mid, out, nonfinite);
    return cudaGetLastError();
}

}  // namespace evsur

extern "C" int sur_gemm(const sur_gemm_args *g, int *d_status, void *stream)
{
    if (!g) return SUR_EINVAL;
    return evsur::gemm(*g, d_status, static_cast<cudaStream_t>(stream));
}

extern "C" int sur_indicators(const float *d_fields, int batch, int H, int W, float rho_mid, double *d_out,
                              void *stream)
{
    if (!d_fields || !d_out || batch < 1 || H < 1 || W < 1) return SUR_EINVAL;
    const cudaError_t e = evsur::indicators(d_fields, batch, (long long)H * W, rho_mid, d_out, nullptr,
                                            static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SUR_OK : SUR_ECUDA;
}
