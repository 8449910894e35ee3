// Learned warm start for the pressure solve: a small 3-level encoder/decoder
// CNN (16/32 channels) on BF16 activations and weights with FP32 accumulation,
// trained on the GPU by these kernels (forward, backward-data,
// backward-weight, loss, Adam).  The network maps (b / s, (1/rho) / max) to
// p / s, s the rms of the mean-free right-hand side; the multigrid solve then
// continues from s * (y - mean y) to the requested residual.
//
// Convolutions are implicit GEMMs on the tensor cores (mma.sync m16n8k16,
// BF16 in, FP32 accumulate): an 8 x 16 output tile (M = 128 pixels) per CTA,
// the input tile with its 1-pixel halo and all weights staged in shared
// memory with padded strides (conflict-free fragment loads), K = 9 taps x
// input channels.  Activations are NHWC with channel counts padded to 16.
// The weight gradient is split over pixel chunks and reduced in a fixed
// order, so training is deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "ib_internal.cuh"

namespace ibk {
namespace {

using bf16 = __nv_bfloat16;
constexpr int CH = 8, CW = 16;  // conv output tile: 8 rows x 16 columns

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// keep each bf16 half of v where the matching half of the mask is > 0
__device__ __forceinline__ uint32_t relu_mask(uint32_t v, uint32_t m)
{
    uint32_t r = 0;
    if ((m & 0x8000u) == 0 && (m & 0x7fffu) != 0) r |= v & 0xffffu;
    if ((m & 0x80000000u) == 0 && (m & 0x7fff0000u) != 0) r |= v & 0xffff0000u;
    return r;
}

template <int CIN, int COUT, bool MASK>
constexpr size_t conv_smem()
{
    return ((size_t)(MASK ? 4 : 2) * (CH + 2) * (CW + 2) * (CIN + 8) + (size_t)COUT * (9 * CIN + 8)) * 2;
}

// 16-byte asynchronous copy (both addresses 16-byte aligned); src-size 0 writes zeros.
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc, bool valid)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
    const int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Address of channels [8q, 8q + 8) of the convolution input at pixel
// (bz, gy, gx) (inside the image).  With CUP > 0 the input is the channel
// concatenation up2(xu) ++ x: channels below CUP come from the half-resolution
// tensor xu (nearest upsampling, CUP channels), the rest from x (CIN - CUP
// channels); the concatenated tensor is never stored.
template <int CIN, int CUP>
__device__ __forceinline__ const bf16 *in_chunk(const bf16 *x, const bf16 *xu, int bz, int H, int W,
                                                int gy, int gx, int q)
{
    if (CUP > 0 && q < CUP / 8)
        return xu + (((long)bz * (H / 2) + gy / 2) * (W / 2) + gx / 2) * CUP + 8 * q;
    return x + (((long)bz * H + gy) * W + gx) * (CIN - CUP) + 8 * q - CUP;
}

// y = act(conv3x3(x * [xmask > 0]) + bias), NHWC, zero padding.
// w: [COUT][9][CIN] (tap = 3 dy + dx multiplies x[i + dy - 1, j + dx - 1]).
// Persistent: each CTA stages all weights once, then walks output tiles of
// 8 x 16 pixels; the next tile (and its mask) is copied into the other
// shared buffer with cp.async while the current one is on the tensor cores.
// CUP > 0: the input is up2(xu) ++ x (see in_chunk).
template <int CIN, int COUT, int CUP, bool MASK>
__global__ void __launch_bounds__(128)
k_conv_fwd(int B, int H, int W, const bf16 *__restrict__ x, const bf16 *__restrict__ xu,
           const bf16 *__restrict__ xmask,
           const bf16 *__restrict__ w, const float *__restrict__ bias, int relu,
           bf16 *__restrict__ y, float *__restrict__ y32)
{
    constexpr int XS = CIN + 8, WS = 9 * CIN + 8, NT = COUT / 8;
    constexpr int TP = (CH + 2) * (CW + 2);       // pixels of a haloed tile
    static_assert(CIN % 16 == 0 && CUP % 8 == 0 && (CUP == 0 || !MASK), "channel layout");
    extern __shared__ __align__(16) unsigned char conv_sm[];
    bf16 *ws = (bf16 *)conv_sm;
    bf16 *xs0 = ws + COUT * WS;                    // 2 input buffers, then 2 mask buffers
    const int tw = (W + CW - 1) / CW, th = (H + CH - 1) / CH, ntiles = B * tw * th;
    for (int k = threadIdx.x; k < COUT * (9 * CIN / 2); k += 128) {
        const int co = k / (9 * CIN / 2), q = k - co * (9 * CIN / 2);
        *(uint32_t *)(ws + co * WS + 2 * q) = *(const uint32_t *)(w + (long)co * 9 * CIN + 2 * q);
    }
    auto issue = [&](int tl, int buf) {
        const int bz = tl / (tw * th), rem = tl - bz * tw * th;
        const int ty0 = (rem / tw) * CH, tx0 = (rem - (rem / tw) * tw) * CW;
        bf16 *xs = xs0 + buf * TP * XS;
        bf16 *ms = xs0 + (2 + buf) * TP * XS;
        for (int k = threadIdx.x; k < TP * (CIN / 8); k += 128) {
            const int pix = k / (CIN / 8), q = k - pix * (CIN / 8);
            const int r = pix / (CW + 2), c = pix - r * (CW + 2);
            const int gy = ty0 + r - 1, gx = tx0 + c - 1;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            cp_async16(xs + pix * XS + 8 * q, in ? in_chunk<CIN, CUP>(x, xu, bz, H, W, gy, gx, q) : x, in);
            if (MASK)
                cp_async16(ms + pix * XS + 8 * q,
                           xmask + (in ? (((long)bz * H + gy) * W + gx) * CIN + 8 * q : 0), in);
        }
        cp_async_commit();
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
    int buf = 0;
    if (blockIdx.x < ntiles) issue(blockIdx.x, 0);
    for (int tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int tn = tl + gridDim.x;
        if (tn < ntiles) { issue(tn, buf ^ 1); cp_async_wait<1>(); }
        else cp_async_wait<0>();
        __syncthreads();
        const bf16 *xs = xs0 + buf * TP * XS;
        const bf16 *ms = xs0 + (2 + buf) * TP * XS;
        float acc[2][NT][4];
#pragma unroll
        for (int a = 0; a < 2; a++)
#pragma unroll
            for (int b = 0; b < NT; b++)
#pragma unroll
                for (int q = 0; q < 4; q++) acc[a][b][q] = 0.0f;
#pragma unroll 1
        for (int tap = 0; tap < 9; tap++) {
            const int dy = tap / 3, dx = tap - 3 * (tap / 3);
#pragma unroll
            for (int c0 = 0; c0 < CIN; c0 += 16) {
                uint32_t bf[NT][2];
#pragma unroll
                for (int nt = 0; nt < NT; nt++) {
                    const bf16 *wp = ws + (nt * 8 + g) * WS + tap * CIN + c0 + 2 * t4;
                    bf[nt][0] = *(const uint32_t *)wp;
                    bf[nt][1] = *(const uint32_t *)(wp + 8);
                }
#pragma unroll
                for (int mt = 0; mt < 2; mt++) {
                    const int r = 2 * warp + mt;
                    const int o0 = ((r + dy) * (CW + 2) + g + dx) * XS + c0 + 2 * t4, o1 = o0 + 8 * XS;
                    uint32_t af[4];
                    af[0] = *(const uint32_t *)(xs + o0);
                    af[1] = *(const uint32_t *)(xs + o1);
                    af[2] = *(const uint32_t *)(xs + o0 + 8);
                    af[3] = *(const uint32_t *)(xs + o1 + 8);
                    if (MASK) {
                        af[0] = relu_mask(af[0], *(const uint32_t *)(ms + o0));
                        af[1] = relu_mask(af[1], *(const uint32_t *)(ms + o1));
                        af[2] = relu_mask(af[2], *(const uint32_t *)(ms + o0 + 8));
                        af[3] = relu_mask(af[3], *(const uint32_t *)(ms + o1 + 8));
                    }
#pragma unroll
                    for (int nt = 0; nt < NT; nt++) mma_bf16(acc[mt][nt], af, bf[nt]);
                }
            }
        }
        const int bz = tl / (tw * th), rem = tl - bz * tw * th;
        const int ty0 = (rem / tw) * CH, tx0 = (rem - (rem / tw) * tw) * CW;
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            const int oy = ty0 + 2 * warp + mt;
            if (oy >= H) continue;
#pragma unroll
            for (int nt = 0; nt < NT; nt++) {
                const int co = nt * 8 + 2 * t4;
                const float b0 = bias ? bias[co] : 0.0f, b1 = bias ? bias[co + 1] : 0.0f;
#pragma unroll
                for (int half = 0; half < 2; half++) {
                    const int ox = tx0 + g + 8 * half;
                    if (ox >= W) continue;
                    float v0 = acc[mt][nt][2 * half] + b0, v1 = acc[mt][nt][2 * half + 1] + b1;
                    if (relu) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                    const long off = (((long)bz * H + oy) * W + ox) * COUT + co;
                    *(__nv_bfloat162 *)(y + off) = __floats2bfloat162_rn(v0, v1);
                    if (y32 && co == 0) y32[off / COUT] = v0;  // channel 0 only
                }
            }
        }
        __syncthreads();  // the buffer just read is refilled by the next issue
        buf ^= 1;
    }
}

// ---- fifth-generation tensor cores (tcgen05) --------------------------
// Shared-memory matrix descriptor of a K-major operand without swizzling:
// core matrices of 8 rows x 16 bytes stored as 128 contiguous bytes; lbo =
// byte distance between core matrices adjacent along K, sbo = along M (or
// N); start, lbo, sbo are multiples of 16 (encoded >> 4); bits 46-47 carry
// the descriptor version (1).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both
// operands K-major, no negation or sparsity: D format bits 4-5 (1 = F32), A
// and B format bits 7-9 and 10-12 (1 = BF16), N >> 3 in bits 17-22, M >> 4
// in bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long cnn_gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the phase of a shared-memory barrier with the given parity: true
// once it has completed, false when limit_ns of global time (or 2^26 polls)
// pass first.
__device__ __forceinline__ bool cnn_mbar_wait(unsigned long long *bar, unsigned parity,
                                              unsigned long long limit_ns)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    const unsigned long long t0 = cnn_gtimer();
    for (int it = 0; it < (1 << 26); it++) {
        unsigned done;
        asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, P;\n}\n" : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (cnn_gtimer() - t0 > limit_ns) return false;
    }
    return false;
}

// Set by a tensor-core convolution whose completion wait ran out (checked by
// the synchronising network calls).
__device__ int g_cnn_fault = 0;

template <int N>
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t *r);
template <>
__device__ __forceinline__ void tmem_ld32<16>(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                 "%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld32<32>(uint32_t taddr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                 "%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,"
                 "%31}, [%32];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                   "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                   "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                   "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

constexpr int kTcPix = 128;              // output pixels of a row segment
constexpr int kTcNP = kTcPix + 2;        // input pixels of a staged row (with halo)

template <int CIN, int COUT>
constexpr size_t conv_tc_smem()
{
    return (size_t)(CIN / 8) * 4 * kTcNP * 16 + (size_t)9 * (CIN / 8) * COUT * 16 + 16;
}

// y = act(conv3x3(x) + bias) on the fifth-generation tensor cores.  A work
// unit is a strip of 128 output pixels (a row segment) over rpu rows;
// each output row is an implicit GEMM D[128 x COUT] = sum over the 9 taps
// and 16-channel chunks of A_tap[128 x 16] B_tap[16 x COUT]
// (tcgen05.mma kind::f16, M = 128, N = COUT, K = 16: BF16 operands from
// shared memory, FP32 accumulators in tensor memory), issued by one thread
// and committed to a shared barrier (bounded wait).  Persistent: a CTA
// allocates its accumulator columns and stages all weights once
// ([tap][8-channel plane][cout][8]), then walks units.  Input rows live in a
// ring of four slots, plane by plane (8 channels a plane, 130 pixels at
// 16-byte steps, zero outside the image; channels below CUP from the
// half-resolution xu, nearest up-sampling, as k_conv_fwd): a unit stages
// its first three rows, then one new row per output row while the tensor
// cores work on the previous one, and a tap's A is the
// slot of row r - 1 + dy shifted by dx pixels, so its core matrices (8
// consecutive pixels x 8 channels) are 128 contiguous bytes, 128 bytes apart
// along M and one plane apart along K.  Each warp reads its 32 accumulator
// lanes (one pixel a thread) and writes bias + ReLU as BF16 NHWC (and the
// FP32 channel 0 when y32 is given).  W must be a multiple of 128.  The
// accumulation order (taps, then 16-channel chunks) is k_conv_fwd's.
template <int CIN, int COUT, int CUP>
__global__ void __launch_bounds__(128)
k_conv_tc(int B, int H, int W, int rpu, const bf16 *__restrict__ x, const bf16 *__restrict__ xu,
          const bf16 *__restrict__ w, const float *__restrict__ bias, int relu,
          bf16 *__restrict__ y, float *__restrict__ y32)
{
    static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32) && CUP % 8 == 0, "shapes");
    constexpr int KP = CIN / 8;                  // 8-channel planes
    constexpr uint32_t SL = kTcNP * 16;          // bytes of a row slot in a plane
    constexpr uint32_t PL = 4 * SL;              // bytes of an input plane (4 slots)
    constexpr uint32_t WPL = COUT * 16;          // bytes of a weight plane
    extern __shared__ __align__(1024) unsigned char tc_sm[];
    unsigned char *xs = tc_sm;
    unsigned char *wsm = tc_sm + KP * PL;
    unsigned long long *mbar = (unsigned long long *)(wsm + 9 * KP * WPL);
    uint32_t *tslot = (uint32_t *)(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int segs = W / kTcPix, bands = (H + rpu - 1) / rpu;
    const int units = B * segs * bands;
    if (warp == 0) {
        // 32 accumulator columns (COUT <= 32), the minimum allocation
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"((unsigned)__cvta_generic_to_shared(tslot)), "r"(32u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n"
                     ::"r"((unsigned)__cvta_generic_to_shared(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    // weights: [tap][plane][cout][8] from [cout][tap][CIN], 16-byte chunks
    for (int k = tid; k < 9 * KP * COUT; k += 128) {
        const int co = k % COUT, rest = k / COUT, k8 = rest % KP, tap = rest / KP;
        const uint4 v = *(const uint4 *)(w + ((long)co * 9 + tap) * CIN + 8 * k8);
        *(uint4 *)(wsm + ((tap * KP + k8) * COUT + co) * 16) = v;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t taddr = *tslot;
    const uint32_t xb = (unsigned)__cvta_generic_to_shared(xs);
    const uint32_t wb = (unsigned)__cvta_generic_to_shared(wsm);
    constexpr uint32_t idesc = umma_idesc_bf16(kTcPix, COUT);
    unsigned phase = 0;
    bool fail = false, stuck = false;
    // input row gy of the strip at x0 into ring slot gy & 3
    auto stage = [&](int bz, int gy, int x0) {
        const int slot = gy & 3;
        for (int k = tid; k < kTcNP * KP; k += 128) {
            const int px = k % kTcNP, k8 = k / kTcNP, gx = x0 - 1 + px;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                v = *(const uint4 *)in_chunk<CIN, CUP>(x, xu, bz, H, W, gy, gx, k8);
            *(uint4 *)(xs + k8 * PL + slot * SL + px * 16) = v;
        }
    };
    for (int u = blockIdx.x; u < units && !fail; u += gridDim.x) {
        const int seg = u % segs, band = (u / segs) % bands, bz = u / (segs * bands);
        const int x0 = seg * kTcPix, r0 = band * rpu, r1 = min(r0 + rpu, H);
        stage(bz, r0 - 1, x0);
        stage(bz, r0, x0);
        stage(bz, r0 + 1, x0);
        for (int row = r0; row < r1; row++) {
            // the operands, written by the generic proxy, are read by the
            // tensor cores through the async proxy
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (tid == 0) {
#pragma unroll 1
                for (int tap = 0; tap < 9; tap++) {
                    const int dy = tap / 3, dx = tap - 3 * (tap / 3);
                    const uint32_t a0 = xb + ((row - 1 + dy) & 3) * SL + dx * 16;
#pragma unroll
                    for (int kc = 0; kc < CIN / 16; kc++) {
                        const uint64_t ad = umma_desc(a0 + 2 * kc * PL, PL, 128);
                        const uint64_t bd = umma_desc(wb + (tap * KP + 2 * kc) * WPL, WPL, 128);
                        const unsigned acc = (tap > 0 || kc > 0) ? 1u : 0u;
                        asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                                     ::"r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                             ::"r"((unsigned)__cvta_generic_to_shared(mbar)) : "memory");
            }
            // the next row's input while the tensor cores work: its slot
            // held row - 2, which no MMA of this row reads
            if (row + 1 < r1) stage(bz, row + 2, x0);
            const bool done = cnn_mbar_wait(mbar, phase, 50000000ull);
            if (__syncthreads_or(!done)) {
                // the MMAs did not complete in 50 ms: report and stop; wait
                // up to 0.5 s more for them before the accumulators are
                // released
                if (tid == 0) atomicExch(&g_cnn_fault, 1);
                stuck = !__syncthreads_and(cnn_mbar_wait(mbar, phase, 500000000ull));
                fail = true;
                break;
            }
            phase ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint32_t acc[COUT];
            tmem_ld32<COUT>(taddr + ((uint32_t)(32 * warp) << 16), acc);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            const long off = (((long)bz * H + row) * W + x0 + 32 * warp + lane) * COUT;
            uint32_t packed[COUT / 2];
#pragma unroll
            for (int c = 0; c < COUT; c += 2) {
                float v0 = __uint_as_float(acc[c]) + bias[c], v1 = __uint_as_float(acc[c + 1]) + bias[c + 1];
                if (relu) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                if (c == 0 && y32) y32[off / COUT] = v0;
                __nv_bfloat162 b2 = __floats2bfloat162_rn(v0, v1);
                packed[c / 2] = *(uint32_t *)&b2;
            }
#pragma unroll
            for (int q = 0; q < COUT / 8; q++)
                *(uint4 *)(y + off + 8 * q) = make_uint4(packed[4 * q], packed[4 * q + 1],
                                                         packed[4 * q + 2], packed[4 * q + 3]);
            // the accumulators are read before the next row's MMAs overwrite
            // them, and the ring slot of row - 1 before it is restaged
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    // MMAs that never completed leave their columns allocated rather than
    // released under them
    if (warp == 0 && !stuck)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(32u));
}

// Partial weight (and bias) gradients of one tap over a chunk of output
// tiles: dW[co][tap][ci] += sum_p g[p][co] x[p + tap][ci], with
// g = gy * [ymask > 0].  M = COUT, N = CIN, K = pixels (16 per step).
template <int CIN, int COUT, int CUP>
__global__ void __launch_bounds__(128)
k_conv_dw(int B, int H, int W, int tiles_per_chunk, const bf16 *__restrict__ x,
          const bf16 *__restrict__ xu, const bf16 *__restrict__ gy, const bf16 *__restrict__ ymask,
          float *__restrict__ part_w, float *__restrict__ part_b)
{
    constexpr int XS = CIN + 8, GS = COUT + 8, MT = COUT / 16, NT = CIN / 8;
    constexpr int FR = MT * NT;                 // fragments per tap
    constexpr int FPW = (FR + 3) / 4;           // fragments per warp
    __shared__ __align__(16) bf16 xs[(CH + 2) * (CW + 2) * XS];
    __shared__ __align__(16) bf16 gs[CH * CW * GS];
    const int tap = blockIdx.x, chunk = blockIdx.y;
    const int dy = tap / 3, dx = tap - 3 * (tap / 3);
    const int tw = (W + CW - 1) / CW, th = (H + CH - 1) / CH, ntiles = B * tw * th;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
    float acc[FPW][4];
#pragma unroll
    for (int f = 0; f < FPW; f++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[f][q] = 0.0f;
    float bacc = 0.0f;  // bias partial of channel threadIdx.x (tap 0 only)
    for (int tl = chunk * tiles_per_chunk; tl < min(ntiles, (chunk + 1) * tiles_per_chunk); tl++) {
        const int bz = tl / (tw * th), rem = tl - bz * tw * th;
        const int ty0 = (rem / tw) * CH, tx0 = (rem - (rem / tw) * tw) * CW;
        __syncthreads();
        for (int k = threadIdx.x; k < (CH + 2) * (CW + 2) * (CIN / 8); k += 128) {
            const int pix = k / (CIN / 8), q = k - pix * (CIN / 8);
            const int r = pix / (CW + 2), c = pix - r * (CW + 2);
            const int yy = ty0 + r - 1, xx = tx0 + c - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = *(const uint4 *)in_chunk<CIN, CUP>(x, xu, bz, H, W, yy, xx, q);
            *(uint4 *)(xs + pix * XS + 8 * q) = v;
        }
        for (int k = threadIdx.x; k < CH * CW * (COUT / 2); k += 128) {
            const int pix = k / (COUT / 2), cp = k - pix * (COUT / 2);
            const int r = pix / CW, c = pix - r * CW;
            const int yy = ty0 + r, xx = tx0 + c;
            uint32_t v = 0;
            if (yy < H && xx < W) {
                const long off = (((long)bz * H + yy) * W + xx) * COUT + 2 * cp;
                v = *(const uint32_t *)(gy + off);
                if (ymask) v = relu_mask(v, *(const uint32_t *)(ymask + off));
            }
            *(uint32_t *)(gs + pix * GS + 2 * cp) = v;
        }
        __syncthreads();
        if (tap == 0 && threadIdx.x < COUT)
            for (int pix = 0; pix < CH * CW; pix++) bacc += __bfloat162float(gs[pix * GS + threadIdx.x]);
#pragma unroll
        for (int f = 0; f < FPW; f++) {
            const int fr = warp * FPW + f;
            if (fr >= FR) break;
            const int mt = fr / NT, nt = fr - mt * NT;
            const int co = mt * 16 + g, ci = nt * 8 + g;
#pragma unroll 2
            for (int r = 0; r < CH; r++) {  // K step = the 16 pixels of output row r
                const bf16 *ga = gs + (r * CW) * GS;
                const int p0 = 2 * t4, p1 = 2 * t4 + 1, p2 = 2 * t4 + 8, p3 = 2 * t4 + 9;
                __nv_bfloat162 a0, a1, a2, a3;
                a0.x = ga[p0 * GS + co];       a0.y = ga[p1 * GS + co];
                a1.x = ga[p0 * GS + co + 8];   a1.y = ga[p1 * GS + co + 8];
                a2.x = ga[p2 * GS + co];       a2.y = ga[p3 * GS + co];
                a3.x = ga[p2 * GS + co + 8];   a3.y = ga[p3 * GS + co + 8];
                uint32_t af[4] = {*(uint32_t *)&a0, *(uint32_t *)&a1, *(uint32_t *)&a2, *(uint32_t *)&a3};
                const bf16 *xb = xs + ((r + dy) * (CW + 2) + dx) * XS + ci;
                __nv_bfloat162 b0, b1;
                b0.x = xb[p0 * XS]; b0.y = xb[p1 * XS];
                b1.x = xb[p2 * XS]; b1.y = xb[p3 * XS];
                uint32_t bf[2] = {*(uint32_t *)&b0, *(uint32_t *)&b1};
                mma_bf16(acc[f], af, bf);
            }
        }
    }
#pragma unroll
    for (int f = 0; f < FPW; f++) {
        const int fr = warp * FPW + f;
        if (fr >= FR) break;
        const int mt = fr / NT, nt = fr - mt * NT;
        // C fragment: rows co (g, g+8), columns ci (2 t4, 2 t4 + 1)
        const int co0 = mt * 16 + g, ci0 = nt * 8 + 2 * t4;
        float *pw = part_w + (long)chunk * COUT * 9 * CIN;
        pw[(long)co0 * 9 * CIN + tap * CIN + ci0] = acc[f][0];
        pw[(long)co0 * 9 * CIN + tap * CIN + ci0 + 1] = acc[f][1];
        pw[(long)(co0 + 8) * 9 * CIN + tap * CIN + ci0] = acc[f][2];
        pw[(long)(co0 + 8) * 9 * CIN + tap * CIN + ci0 + 1] = acc[f][3];
    }
    if (tap == 0 && threadIdx.x < COUT) part_b[(long)chunk * COUT + threadIdx.x] = bacc;
}

// Sum of the chunk partials in chunk order.
__global__ void k_reduce_parts(int nchunks, long n, const float *__restrict__ part,
                               float *__restrict__ out)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float s = 0.0f;
    for (int c = 0; c < nchunks; c++) s += part[(long)c * n + k];
    out[k] = s;
}

// --- layout helpers (bf16 NHWC) -----------------------------------------
__global__ void k_pool2(long nout, int H2, int W2, int C, const bf16 *__restrict__ x,
                        bf16 *__restrict__ y)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nout) return;
    const int c = (int)(k % C);
    long p = k / C;
    const int j = (int)(p % W2);
    p /= W2;
    const int i = (int)(p % H2);
    const long b = p / H2;
    const int W = 2 * W2;
    const long base = ((b * (2 * H2) + 2 * i) * W + 2 * j) * C + c;
    float s = __bfloat162float(x[base]) + __bfloat162float(x[base + C]) +
              __bfloat162float(x[base + (long)W * C]) + __bfloat162float(x[base + (long)W * C + C]);
    y[k] = __float2bfloat16_rn(0.25f * s);
}

// gt = sum over 2x2 of g[..., :C1];  gs = g[..., C1:] (+ gs_add)
__global__ void k_up_cat_bwd(long nhalf, int H2, int W2, int C1, int C2, const bf16 *__restrict__ g,
                             bf16 *__restrict__ gt)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nhalf) return;
    const int c = (int)(k % C1);
    long p = k / C1;
    const int j = (int)(p % W2);
    p /= W2;
    const int i = (int)(p % H2);
    const long b = p / H2;
    const int W = 2 * W2, C = C1 + C2;
    const long base = ((b * (2 * H2) + 2 * i) * W + 2 * j) * C + c;
    float s = __bfloat162float(g[base]) + __bfloat162float(g[base + C]) +
              __bfloat162float(g[base + (long)W * C]) + __bfloat162float(g[base + (long)W * C + C]);
    gt[k] = __float2bfloat16_rn(s);
}

// gskip = g_cat[..., C1:] + pool2_bwd(gp)   (gp at half resolution, C2 channels)
__global__ void k_skip_grad(long n, int H, int W, int C1, int C2, const bf16 *__restrict__ gcat,
                            const bf16 *__restrict__ gp, bf16 *__restrict__ gskip)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int c = (int)(k % C2);
    long p = k / C2;
    const int j = (int)(p % W);
    p /= W;
    const int i = (int)(p % H);
    const long b = p / H;
    float v = __bfloat162float(gcat[((b * H + i) * W + j) * (C1 + C2) + C1 + c]);
    v += 0.25f * __bfloat162float(gp[((b * (H / 2) + i / 2) * (W / 2) + j / 2) * C2 + c]);
    gskip[k] = __float2bfloat16_rn(v);
}

// --- features, loss, output ----------------------------------------------
// Per-sample statistics of the network input, in two launches: partial sums
// over kRedBlocks CTAs per sample, then a fixed-order fold.  One pass gives
// sum (b - b0) and sum (b - b0)^2 with b0 the sample's first value (a shift
// that keeps the variance free of cancellation), and min rho (max(1/rho) is
// 1/min(rho) exactly, IEEE division being monotone).
// stats[kStat * smp + ...]: 0 mean b, 1 s = rms(b - mean) (1 if zero),
// 2 1/s, 3 min rho, 4 1/(s pscale), 5 mean of the network output.
constexpr int kRedBlocks = 256, kStat = 8;

__device__ __forceinline__ void block_fold3(double (*sh)[256], double &a, double &b, double &c, bool cmin)
{
    sh[0][threadIdx.x] = a; sh[1][threadIdx.x] = b; sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
            sh[2][threadIdx.x] = cmin ? fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + o])
                                      : sh[2][threadIdx.x] + sh[2][threadIdx.x + o];
        }
        __syncthreads();
    }
    a = sh[0][0]; b = sh[1][0]; c = sh[2][0];
}

__global__ void __launch_bounds__(256)
k_stats_part(int N2, const double *__restrict__ b, const double *__restrict__ rho,
             double *__restrict__ part)
{
    __shared__ double sh[3][256];
    const int smp = blockIdx.y;
    const double *bb = b + (long)smp * N2, *rr = rho + (long)smp * N2;
    const double b0 = bb[0];
    double sd = 0.0, sq = 0.0, mn = INFINITY;
    for (int k = blockIdx.x * 256 + threadIdx.x; k < N2; k += 256 * kRedBlocks) {
        const double d = bb[k] - b0;
        sd += d; sq += d * d; mn = fmin(mn, rr[k]);
    }
    block_fold3(sh, sd, sq, mn, true);
    if (threadIdx.x == 0) {
        double *o = part + ((long)smp * kRedBlocks + blockIdx.x) * 3;
        o[0] = sd; o[1] = sq; o[2] = mn;
    }
}

__global__ void __launch_bounds__(256)
k_stats_final(int N2, const double *__restrict__ b, const double *__restrict__ part, double pscale,
              double *__restrict__ stats)
{
    __shared__ double sh[3][256];
    const int smp = blockIdx.x;
    double sd = 0.0, sq = 0.0, mn = INFINITY;
    if (threadIdx.x < kRedBlocks) {
        const double *o = part + ((long)smp * kRedBlocks + threadIdx.x) * 3;
        sd = o[0]; sq = o[1]; mn = o[2];
    }
    block_fold3(sh, sd, sq, mn, true);
    if (threadIdx.x == 0) {
        const double md = sd / N2, var = fmax(sq / N2 - md * md, 0.0), r = sqrt(var);
        const double sc = r > 0.0 ? r : 1.0;
        double *st = stats + kStat * smp;
        st[0] = b[(long)smp * N2] + md;
        st[1] = sc;
        st[2] = 1.0 / sc;
        st[3] = mn;
        st[4] = 1.0 / (sc * pscale);
    }
}

// Mean of the network output per sample (partials, then the fold into stats[5]).
__global__ void __launch_bounds__(256)
k_ysum_part(int N2, const float *__restrict__ y32, double *__restrict__ part)
{
    __shared__ double sh[3][256];
    const int smp = blockIdx.y;
    const float *yy = y32 + (long)smp * N2;
    double s = 0.0, z0 = 0.0, z1 = 0.0;
    for (int k = blockIdx.x * 256 + threadIdx.x; k < N2; k += 256 * kRedBlocks) s += (double)yy[k];
    block_fold3(sh, s, z0, z1, false);
    if (threadIdx.x == 0) part[(long)smp * kRedBlocks + blockIdx.x] = s;
}

__global__ void __launch_bounds__(256)
k_ymean_final(int N2, const double *__restrict__ part, double *__restrict__ stats)
{
    __shared__ double sh[3][256];
    double s = threadIdx.x < kRedBlocks ? part[(long)blockIdx.x * kRedBlocks + threadIdx.x] : 0.0;
    double z0 = 0.0, z1 = 0.0;
    block_fold3(sh, s, z0, z1, false);
    if (threadIdx.x == 0) stats[kStat * blockIdx.x + 5] = s / N2;
}

// x[..., 0] = (b - mean)/s, x[..., 1] = (1/rho)/max(1/rho) = min(rho)/rho,
// other channels 0 (BF16, rounded from FP32); and (training)
// t = p / (s pscale), pscale = h^2 c.
__global__ void k_features(long n, int N2, const double *__restrict__ b, const double *__restrict__ rho,
                           const double *__restrict__ p, const double *__restrict__ stats,
                           bf16 *__restrict__ x, float *__restrict__ t)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double *st = stats + kStat * (k / N2);
    const float f0 = (float)((b[k] - st[0]) * st[2]);
    const float f1 = (float)st[3] / (float)rho[k];
    __nv_bfloat162 v = __floats2bfloat162_rn(f0, f1);
    uint32_t *xp = (uint32_t *)(x + k * 16);
    xp[0] = *(uint32_t *)&v;
#pragma unroll
    for (int q = 1; q < 8; q++) xp[q] = 0u;
    if (t) t[k] = (float)(p[k] * st[4]);
}

// Mean-removed squared error per sample (one CTA per sample): loss partial and
// the gradient 2 d / (B n) minus its mean, written as BF16 channel 0 of a
// 16-channel tensor.
__global__ void __launch_bounds__(256)
k_loss(int N2, int Bn, const float *__restrict__ y32, const float *__restrict__ t,
       bf16 *__restrict__ gy, float *__restrict__ lsum)
{
    __shared__ float sh[2][256];
    const long base = (long)blockIdx.x * N2;
    float sy = 0.0f, st = 0.0f;
    for (int k = threadIdx.x; k < N2; k += 256) { sy += y32[base + k]; st += t[base + k]; }
    sh[0][threadIdx.x] = sy; sh[1][threadIdx.x] = st;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) { sh[0][threadIdx.x] += sh[0][threadIdx.x + o]; sh[1][threadIdx.x] += sh[1][threadIdx.x + o]; }
        __syncthreads();
    }
    const float my = sh[0][0] / N2, mt = sh[1][0] / N2;
    __syncthreads();
    float l = 0.0f, gs = 0.0f;
    const float sc = 2.0f / ((float)Bn * (float)N2);
    for (int k = threadIdx.x; k < N2; k += 256) {
        float d = (y32[base + k] - my) - (t[base + k] - mt);
        l += d * d;
        gs += sc * d;
    }
    sh[0][threadIdx.x] = l; sh[1][threadIdx.x] = gs;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) { sh[0][threadIdx.x] += sh[0][threadIdx.x + o]; sh[1][threadIdx.x] += sh[1][threadIdx.x + o]; }
        __syncthreads();
    }
    const float gmean = sh[1][0] / N2;
    for (int k = threadIdx.x; k < N2; k += 256) {
        float d = (y32[base + k] - my) - (t[base + k] - mt);
        uint32_t *gp = (uint32_t *)(gy + (base + k) * 16);
        __nv_bfloat162 v = __floats2bfloat162_rn(sc * d - gmean, 0.0f);
        gp[0] = *(uint32_t *)&v;
#pragma unroll
        for (int q = 1; q < 8; q++) gp[q] = 0u;
    }
    if (threadIdx.x == 0) lsum[blockIdx.x] = sh[0][0] / ((float)Bn * (float)N2);
}

// p0 = s pscale (y - mean y), FP64 out.
__global__ void k_output(long n, int N2, const float *__restrict__ y32, const double *__restrict__ stats,
                         double pscale, double *__restrict__ p0)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double *st = stats + kStat * (k / N2);
    p0[k] = st[1] * pscale * ((double)y32[k] - st[5]);
}

// 2x2 mean of B samples of (2 Nc) x (2 Nc) into Nc x Nc.
__global__ void k_restrict2(long nc, int Nc, const double *__restrict__ in, double *__restrict__ out)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const long N2c = (long)Nc * Nc, smp = k / N2c;
    const int r = (int)(k - smp * N2c), J = r / Nc, I = r - J * Nc, N = 2 * Nc;
    const double *a = in + smp * 4 * N2c + (long)(2 * J) * N + 2 * I;
    out[k] = 0.25 * (a[0] + a[1] + a[N] + a[N + 1]);
}

// Cell-centred bilinear interpolation (9, 3, 3, 1)/16 of Nc x Nc samples to
// (2 Nc) x (2 Nc), zero-gradient at the walls.
__global__ void k_prolong2(long nf, int Nc, const double *__restrict__ ec, double *__restrict__ ef)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const int N = 2 * Nc;
    const long N2 = (long)N * N, smp = k / N2;
    const int r = (int)(k - smp * N2), j = r / N, i = r - j * N;
    const int I = i >> 1, J = j >> 1;
    const int I2 = min(max(I + ((i & 1) ? 1 : -1), 0), Nc - 1);
    const int J2 = min(max(J + ((j & 1) ? 1 : -1), 0), Nc - 1);
    const double *c = ec + smp * (long)Nc * Nc;
    ef[k] = (9.0 * c[J * Nc + I] + 3.0 * c[J * Nc + I2] + 3.0 * c[J2 * Nc + I] + c[J2 * Nc + I2]) *
            0.0625;
}

// Adam with bias correction on FP32 master weights.
__global__ void k_adam(long n, float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.0f - b1) * gk, vk = b2 * v[k] + (1.0f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Master [co][3][3][ci] FP32 -> forward BF16 [COP][9][CIP] (zero padded) and
// backward-data BF16 [CIP][9][COP] with the taps flipped.
__global__ void k_pack(int ci, int co, int cip, int cop, const float *__restrict__ w,
                       bf16 *__restrict__ wf, bf16 *__restrict__ wb)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cop * 9 * cip) return;
    const int o = k / (9 * cip), r = k - o * 9 * cip, tap = r / cip, i = r - tap * cip;
    const float v = (o < co && i < ci) ? w[((long)o * 9 + tap) * ci + i] : 0.0f;
    wf[k] = __float2bfloat16_rn(v);
    if (wb) wb[((long)i * 9 + (8 - tap)) * cop + o] = __float2bfloat16_rn(v);
}

// Padded gradients [COP][9][CIP] and [COP] -> master layout [co][9][ci], [co].
__global__ void k_unpack_grad(int ci, int co, int cip, const float *__restrict__ gpw,
                              const float *__restrict__ gpb, float *__restrict__ gw,
                              float *__restrict__ gb)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < co) gb[k] = gpb[k];
    if (k >= co * 9 * ci) return;
    const int o = k / (9 * ci), r = k - o * 9 * ci, tap = r / ci, i = r - tap * ci;
    gw[k] = gpw[((long)o * 9 + tap) * cip + i];
}

}  // namespace

// rms of (a - mean a) of each sample (one CTA per sample, fixed order: the
// mean first, then the squared deviations).
__global__ void __launch_bounds__(256) k_sample_rms(int N2, const double *__restrict__ a,
                                                    double *__restrict__ out)
{
    __shared__ double sh[256];
    const double *x = a + (long)blockIdx.x * N2;
    double t = 0.0;
    for (int k = threadIdx.x; k < N2; k += 256) t += x[k];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double m = sh[0] / N2;
    __syncthreads();
    double q = 0.0;
    for (int k = threadIdx.x; k < N2; k += 256) {
        const double d = x[k] - m;
        q += d * d;
    }
    sh[threadIdx.x] = q;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(sh[0] / N2);
}

// Mini-batch gather: sample idx[i] of each set into slot i.
__global__ void k_gather3(long n, int N2, const int *__restrict__ idx, const double *__restrict__ a,
                          const double *__restrict__ b, const double *__restrict__ c,
                          double *__restrict__ ga, double *__restrict__ gb, double *__restrict__ gc)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long src = (long)idx[k / N2] * N2 + k % N2;
    ga[k] = a[src];
    gb[k] = b[src];
    gc[k] = c[src];
}

// The batch loss (sum of the per-sample partials, in order) into out.
__global__ void k_loss_record(int B, const float *__restrict__ lsum, float *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    float t = 0.0f;
    for (int b = 0; b < B; b++) t += lsum[b];
    *out = t;
}

// ======================================================================= host
struct CnnLayer {
    int ci, co, cip, cop;     // real and padded channel counts
    bool relu;
    size_t woff, boff;        // offsets in the flat FP32 parameter vector
    size_t pwoff, pboff;      // offsets of the padded gradients [COP][9][CIP], [COP]
    bf16 *wf = nullptr, *wb = nullptr;
};

struct Cnn {
    int c1 = 16, c2 = 32;
    std::vector<CnnLayer> L;
    size_t nparam = 0, npad = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // flat FP32
    void *wmem = nullptr;
    int step = 0;
    int tc = 1;               // forward convolutions on tcgen05: 0 none, 1 where faster, 2 all that fit
    double out_scale = 1.0;   // c in the pressure scale s h^2 c
    // activation workspace, sized for B x N x N
    int capB = 0, capN = 0;
    void *amem = nullptr;
    bf16 *x = nullptr, *a1 = nullptr, *s1 = nullptr, *p1 = nullptr, *a2 = nullptr, *s2 = nullptr,
         *p2 = nullptr, *a3 = nullptr, *t3 = nullptr, *t4 = nullptr,
         *a5 = nullptr, *y = nullptr, *gbig = nullptr, *gbig2 = nullptr,
         *gmid = nullptr, *gmid2 = nullptr, *gsmall = nullptr, *gsmall2 = nullptr, *gcat = nullptr,
         *gup = nullptr;
    float *y32 = nullptr, *t = nullptr, *lsum = nullptr, *gpad = nullptr, *part = nullptr;
    double *stats = nullptr, *rpart = nullptr;
    size_t part_cap = 0;
    // coarse-grid inference: restricted inputs and prolongated outputs
    double *cbuf = nullptr;
    size_t cbuf_cap = 0;
};

namespace {

int g_sms = 0;

// tc: 0 the warp-level kernel; 1 tcgen05 for the shapes where it measured
// faster than the warp-level kernel (16 -> 32 channels: 8.7 against 12.2 us
// at 128^2; the others are bound by operand staging and latency, where the
// warp-level kernel's double-buffered 8 x 16 tiles stage less per output);
// 2 tcgen05 wherever the width is a multiple of 128.
template <int CIN, int COUT, int CUP, bool MASK>
void conv_launch(int B, int H, int W, const bf16 *x, const bf16 *xu, const bf16 *xmask, const bf16 *w,
                 const float *bias, int relu, bf16 *y, float *y32, cudaStream_t s, int tc = 0)
{
    if constexpr (!MASK && (COUT == 16 || COUT == 32)) {
        const bool faster = CIN == 16 && COUT == 32 && CUP == 0;
        if ((tc == 2 || (tc == 1 && faster)) && W % kTcPix == 0) {
            constexpr size_t smt = conv_tc_smem<CIN, COUT>();
            static bool attr_tc = false;
            if (!attr_tc) {
                cudaFuncSetAttribute(k_conv_tc<CIN, COUT, CUP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smt);
                attr_tc = true;
            }
            if (!g_sms) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
                if (g_sms <= 0) g_sms = 152;
            }
            // rows per unit: as many as keep every SM busy, up to 8 (a unit
            // stages rpu + 2 input rows for rpu output rows); CTAs per SM by
            // shared memory (at most 8: 256 of the 512 tensor-memory columns)
            const int per_sm = std::max(1, std::min(8, (int)((227 * 1024) / smt)));
            const long rows = (long)B * H * (W / kTcPix);
            const int rpu = (int)std::max(1L, std::min(std::min((long)H, 8L), rows / g_sms));
            const long units = (long)B * (W / kTcPix) * ((H + rpu - 1) / rpu);
            const int grid = (int)std::min(units, (long)g_sms * per_sm);
            note_launch();
            k_conv_tc<CIN, COUT, CUP><<<grid, 128, smt, s>>>(B, H, W, rpu, x, xu, w, bias, relu, y, y32);
            return;
        }
    }
    constexpr size_t sm = conv_smem<CIN, COUT, MASK>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_conv_fwd<CIN, COUT, CUP, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 152;
    }
    const int ntiles = B * (int)cdiv(W, CW) * (int)cdiv(H, CH);
    const int per_sm = sm <= 56 * 1024 ? 4 : (sm <= 75 * 1024 ? 3 : 2);
    const int grid = std::min(ntiles, g_sms * per_sm);
    note_launch();
    k_conv_fwd<CIN, COUT, CUP, MASK><<<grid, 128, sm, s>>>(B, H, W, x, xu, xmask, w, bias, relu, y, y32);
}

template <int CIN, int COUT>
void conv_fwd(int B, int H, int W, const bf16 *x, const bf16 *xmask, const bf16 *w,
              const float *bias, int relu, bf16 *y, float *y32, cudaStream_t s, int tc = 0)
{
    if (xmask) conv_launch<CIN, COUT, 0, true>(B, H, W, x, nullptr, xmask, w, bias, relu, y, y32, s);
    else conv_launch<CIN, COUT, 0, false>(B, H, W, x, nullptr, xmask, w, bias, relu, y, y32, s, tc);
}

// Convolution of the concatenation up2(xu) ++ x (CUP channels from xu).
template <int CIN, int COUT, int CUP>
void conv_fwd_cat(int B, int H, int W, const bf16 *xu, const bf16 *x, const bf16 *w,
                  const float *bias, int relu, bf16 *y, cudaStream_t s, int tc = 0)
{
    conv_launch<CIN, COUT, CUP, false>(B, H, W, x, xu, nullptr, w, bias, relu, y, nullptr, s, tc);
}

template <int CIN, int COUT, int CUP = 0>
void conv_dw(Cnn &n, int B, int H, int W, const bf16 *x, const bf16 *gy, const bf16 *ymask,
             float *gw_pad, float *gb, cudaStream_t s, const bf16 *xu = nullptr)
{
    const int ntiles = B * (int)cdiv(W, CW) * (int)cdiv(H, CH);
    const int nchunks = std::min(ntiles, 64);
    const int tpc = (ntiles + nchunks - 1) / nchunks;
    float *pw = n.part, *pb = n.part + (size_t)nchunks * COUT * 9 * CIN;
    dim3 g(9, nchunks);
    note_launch();
    k_conv_dw<CIN, COUT, CUP><<<g, 128, 0, s>>>(B, H, W, tpc, x, xu, gy, ymask, pw, pb);
    const long nw = (long)COUT * 9 * CIN;
    note_launch();
    k_reduce_parts<<<cdiv(nw, 256), 256, 0, s>>>(nchunks, nw, pw, gw_pad);
    note_launch();
    k_reduce_parts<<<1, 256, 0, s>>>(nchunks, COUT, pb, gb);
}

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

Cnn *cnn_new(int c1, int c2, unsigned long long seed, cudaStream_t s, cudaError_t *err)
{
    (void)s;
    Cnn *n = new Cnn();
    n->c1 = c1;
    n->c2 = c2;
    auto pad = [](int c) { return (c + 15) / 16 * 16; };
    const int spec[9][3] = {{2, c1, 1}, {c1, c1, 1}, {c1, c2, 1}, {c2, c2, 1}, {c2, c2, 1},
                            {c2, c2, 1}, {2 * c2, c2, 1}, {c2 + c1, c1, 1}, {c1, 1, 0}};
    size_t off = 0;
    for (auto &sp : spec) {
        CnnLayer l;
        l.ci = sp[0]; l.co = sp[1]; l.relu = sp[2] != 0;
        l.cip = pad(l.ci); l.cop = pad(l.co);
        l.woff = off; off += (size_t)l.co * 9 * l.ci;
        l.boff = off; off += (size_t)l.co;
        n->L.push_back(l);
    }
    n->nparam = off;
    size_t po = 0;
    for (auto &l : n->L) {
        l.pwoff = po; po += (size_t)l.cop * 9 * l.cip;
        l.pboff = po; po += (size_t)l.cop;
    }
    n->npad = po;
    size_t bytes = al(off * 4) * 4;
    for (auto &l : n->L) bytes += 2 * al((size_t)l.cop * 9 * l.cip * 2);
    *err = cudaMalloc(&n->wmem, bytes);
    if (*err != cudaSuccess) { n->wmem = nullptr; cnn_free(n); return nullptr; }
    char *q = (char *)n->wmem;
    auto take = [&](size_t b) { char *r = q; q += al(b); return (void *)r; };
    n->w = (float *)take(off * 4); n->m = (float *)take(off * 4);
    n->v = (float *)take(off * 4); n->g = (float *)take(off * 4);
    for (auto &l : n->L) {
        l.wf = (bf16 *)take((size_t)l.cop * 9 * l.cip * 2);
        l.wb = (bf16 *)take((size_t)l.cop * 9 * l.cip * 2);
    }
    // He-normal initial weights (Box-Muller on a splitmix64 stream), zero biases
    std::vector<float> h(off, 0.0f);
    unsigned long long st = seed ^ 0x9E3779B97F4A7C15ULL;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ULL;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    for (auto &l : n->L) {
        const double sd = sqrt(2.0 / (9.0 * l.ci));
        for (size_t k = 0; k < (size_t)l.co * 9 * l.ci; k++) {
            double u1 = next(), u2 = next();
            if (u1 < 1e-300) u1 = 1e-300;
            h[l.woff + k] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
        }
    }
    *err = cudaMemcpy(n->w, h.data(), off * 4, cudaMemcpyHostToDevice);
    if (*err == cudaSuccess) *err = cudaMemset(n->m, 0, off * 4 * 3);
    if (*err != cudaSuccess) { cnn_free(n); return nullptr; }
    return n;
}

void cnn_free(Cnn *n)
{
    if (!n) return;
    if (n->wmem) cudaFree(n->wmem);
    if (n->amem) cudaFree(n->amem);
    if (n->cbuf) cudaFree(n->cbuf);
    delete n;
}

cudaError_t cnn_pack(Cnn &n, cudaStream_t s)
{
    for (auto &l : n.L) {
        int tot = l.cop * 9 * l.cip;
        note_launch();
        k_pack<<<cdiv(tot, 256), 256, 0, s>>>(l.ci, l.co, l.cip, l.cop, n.w + l.woff, l.wf, l.wb);
    }
    return cudaGetLastError();
}

cudaError_t cnn_workspace(Cnn &n, int B, int N)
{
    if (B <= n.capB && N <= n.capN && n.amem) return cudaSuccess;
    if (n.amem) cudaFree(n.amem);
    n.amem = nullptr;
    const size_t P = (size_t)B * N * N, P2 = P / 4, P4 = P / 16;
    const int c1 = n.c1, c2 = n.c2;
    size_t bytes = al(P * 16 * 2) +                       // x
                   al(P * c1 * 2) * 2 +                    // a1, s1
                   al(P2 * c1 * 2) + al(P2 * c2 * 2) * 2 + // p1, a2, s2
                   al(P4 * c2 * 2) * 3 +                   // p2, a3, t3
                   al(P2 * c2 * 2) +                       // t4
                   al(P * c1 * 2) + al(P * 16 * 2) +       // a5, y
                   al(P * 64 * 2) * 2 + al(P2 * 64 * 2) * 2 + al(P4 * 64 * 2) * 2 +  // grads
                   al(P * 64 * 2) + al(P2 * 64 * 2) +      // gcat, gup
                   al(P * 4) + al(P * 4) + al(B * 4) + al(n.npad * 4) + al(B * kStat * 8) +
                   al(B * kRedBlocks * 3 * 8);
    const size_t part = (size_t)64 * (64 * 9 * 64 + 64);
    bytes += al(part * 4);
    cudaError_t e = cudaMalloc(&n.amem, bytes);
    if (e != cudaSuccess) { n.amem = nullptr; return e; }
    char *q = (char *)n.amem;
    auto take = [&](size_t b) { char *r = q; q += al(b); return (void *)r; };
    n.x = (bf16 *)take(P * 16 * 2);
    n.a1 = (bf16 *)take(P * c1 * 2); n.s1 = (bf16 *)take(P * c1 * 2);
    n.p1 = (bf16 *)take(P2 * c1 * 2); n.a2 = (bf16 *)take(P2 * c2 * 2); n.s2 = (bf16 *)take(P2 * c2 * 2);
    n.p2 = (bf16 *)take(P4 * c2 * 2); n.a3 = (bf16 *)take(P4 * c2 * 2); n.t3 = (bf16 *)take(P4 * c2 * 2);
    n.t4 = (bf16 *)take(P2 * c2 * 2);
    n.a5 = (bf16 *)take(P * c1 * 2);
    n.y = (bf16 *)take(P * 16 * 2);
    n.gbig = (bf16 *)take(P * 64 * 2); n.gbig2 = (bf16 *)take(P * 64 * 2);
    n.gmid = (bf16 *)take(P2 * 64 * 2); n.gmid2 = (bf16 *)take(P2 * 64 * 2);
    n.gsmall = (bf16 *)take(P4 * 64 * 2); n.gsmall2 = (bf16 *)take(P4 * 64 * 2);
    n.gcat = (bf16 *)take(P * 64 * 2); n.gup = (bf16 *)take(P2 * 64 * 2);
    n.y32 = (float *)take(P * 4); n.t = (float *)take(P * 4); n.lsum = (float *)take(B * 4);
    n.gpad = (float *)take(n.npad * 4);
    n.stats = (double *)take(B * kStat * 8);
    n.rpart = (double *)take(B * kRedBlocks * 3 * 8);
    n.part = (float *)take(part * 4);
    n.part_cap = part;
    n.capB = B;
    n.capN = N;
    return cudaSuccess;
}

// Forward pass on B samples of N x N (N a multiple of 4).  Fills the
// activation workspace; y32 holds the FP32 output (one channel).
void cnn_forward(Cnn &n, int B, int N, double h, const double *rhs, const double *rho,
                 const double *p, cudaStream_t s)
{
    const int N2 = N * N, H2 = N / 2, H4 = N / 4;
    const long P = (long)B * N2;
    note_launch();
    k_stats_part<<<dim3(kRedBlocks, B), 256, 0, s>>>(N2, rhs, rho, n.rpart);
    note_launch();
    k_stats_final<<<B, 256, 0, s>>>(N2, rhs, n.rpart, h * h * n.out_scale, n.stats);
    note_launch();
    k_features<<<cdiv(P, 256), 256, 0, s>>>(P, N2, rhs, rho, p, n.stats, n.x, p ? n.t : nullptr);
    auto &L = n.L;
    auto bias = [&](int k) { return n.w + L[k].boff; };
    const int tc = n.tc;
    conv_fwd<16, 16>(B, N, N, n.x, nullptr, L[0].wf, bias(0), 1, n.a1, nullptr, s, tc);
    conv_fwd<16, 16>(B, N, N, n.a1, nullptr, L[1].wf, bias(1), 1, n.s1, nullptr, s, tc);
    note_launch();
    k_pool2<<<cdiv((long)B * H2 * H2 * 16, 256), 256, 0, s>>>((long)B * H2 * H2 * 16, H2, H2, 16, n.s1, n.p1);
    conv_fwd<16, 32>(B, H2, H2, n.p1, nullptr, L[2].wf, bias(2), 1, n.a2, nullptr, s, tc);
    conv_fwd<32, 32>(B, H2, H2, n.a2, nullptr, L[3].wf, bias(3), 1, n.s2, nullptr, s, tc);
    note_launch();
    k_pool2<<<cdiv((long)B * H4 * H4 * 32, 256), 256, 0, s>>>((long)B * H4 * H4 * 32, H4, H4, 32, n.s2, n.p2);
    conv_fwd<32, 32>(B, H4, H4, n.p2, nullptr, L[4].wf, bias(4), 1, n.a3, nullptr, s, tc);
    conv_fwd<32, 32>(B, H4, H4, n.a3, nullptr, L[5].wf, bias(5), 1, n.t3, nullptr, s, tc);
    conv_fwd_cat<64, 32, 32>(B, H2, H2, n.t3, n.s2, L[6].wf, bias(6), 1, n.t4, s, tc);  // up2(t3) ++ s2
    conv_fwd_cat<48, 16, 32>(B, N, N, n.t4, n.s1, L[7].wf, bias(7), 1, n.a5, s, tc);     // up2(t4) ++ s1
    conv_fwd<16, 16>(B, N, N, n.a5, nullptr, L[8].wf, bias(8), 0, n.y, n.y32, s, tc);
}

// Loss and gradients of every parameter (into n.g, master layout).
void cnn_backward(Cnn &n, int B, int N, cudaStream_t s)
{
    const int N2 = N * N, H2 = N / 2, H4 = N / 4;
    const long P = (long)B * N2;
    auto &L = n.L;
    note_launch();
    k_loss<<<B, 256, 0, s>>>(N2, B, n.y32, n.t, n.gbig, n.lsum);
    float *gp = n.gpad;
    auto dwb = [&](int k) { return std::make_pair(gp + L[k].pwoff, gp + L[k].pboff); };
    auto unpack = [&](int k) {
        const int tot = std::max(L[k].co * 9 * L[k].ci, L[k].co);
        note_launch();
        k_unpack_grad<<<cdiv(tot, 256), 256, 0, s>>>(L[k].ci, L[k].co, L[k].cip, gp + L[k].pwoff,
                                                    gp + L[k].pboff, n.g + L[k].woff, n.g + L[k].boff);
    };
    // c6 (linear): input a5, grad gbig (16 ch, channel 0)
    conv_dw<16, 16>(n, B, N, N, n.a5, n.gbig, nullptr, dwb(8).first, dwb(8).second, s);
    conv_fwd<16, 16>(B, N, N, n.gbig, nullptr, L[8].wb, nullptr, 0, n.gbig2, nullptr, s);  // grad a5
    // c5: out a5 (mask), in up2(t4) ++ s1
    conv_dw<48, 16, 32>(n, B, N, N, n.s1, n.gbig2, n.a5, dwb(7).first, dwb(7).second, s, n.t4);
    conv_fwd<16, 48>(B, N, N, n.gbig2, n.a5, L[7].wb, nullptr, 0, n.gcat, nullptr, s);     // grad of up2(t4) ++ s1
    note_launch();
    k_up_cat_bwd<<<cdiv((long)B * H2 * H2 * 32, 256), 256, 0, s>>>((long)B * H2 * H2 * 32, H2, H2, 32, 16, n.gcat, n.gmid);  // grad t4
    // c4: out t4 (mask), in up2(t3) ++ s2
    conv_dw<64, 32, 32>(n, B, H2, H2, n.s2, n.gmid, n.t4, dwb(6).first, dwb(6).second, s, n.t3);
    conv_fwd<32, 64>(B, H2, H2, n.gmid, n.t4, L[6].wb, nullptr, 0, n.gup, nullptr, s);     // grad of up2(t3) ++ s2
    note_launch();
    k_up_cat_bwd<<<cdiv((long)B * H4 * H4 * 32, 256), 256, 0, s>>>((long)B * H4 * H4 * 32, H4, H4, 32, 32, n.gup, n.gsmall);  // grad t3
    // c3b: out t3, in a3
    conv_dw<32, 32>(n, B, H4, H4, n.a3, n.gsmall, n.t3, dwb(5).first, dwb(5).second, s);
    conv_fwd<32, 32>(B, H4, H4, n.gsmall, n.t3, L[5].wb, nullptr, 0, n.gsmall2, nullptr, s);  // grad a3
    // c3a: out a3, in p2
    conv_dw<32, 32>(n, B, H4, H4, n.p2, n.gsmall2, n.a3, dwb(4).first, dwb(4).second, s);
    conv_fwd<32, 32>(B, H4, H4, n.gsmall2, n.a3, L[4].wb, nullptr, 0, n.gsmall, nullptr, s);  // grad p2
    // grad s2 = skip part of the c4 input grad + pool2 backward
    note_launch();
    k_skip_grad<<<cdiv((long)B * H2 * H2 * 32, 256), 256, 0, s>>>((long)B * H2 * H2 * 32, H2, H2, 32, 32, n.gup, n.gsmall, n.gmid2);
    // c2b: out s2, in a2
    conv_dw<32, 32>(n, B, H2, H2, n.a2, n.gmid2, n.s2, dwb(3).first, dwb(3).second, s);
    conv_fwd<32, 32>(B, H2, H2, n.gmid2, n.s2, L[3].wb, nullptr, 0, n.gmid, nullptr, s);   // grad a2
    // c2a: out a2, in p1
    conv_dw<16, 32>(n, B, H2, H2, n.p1, n.gmid, n.a2, dwb(2).first, dwb(2).second, s);
    conv_fwd<32, 16>(B, H2, H2, n.gmid, n.a2, L[2].wb, nullptr, 0, n.gmid2, nullptr, s);   // grad p1
    // grad s1 = skip part of the c5 input grad + pool2 backward
    note_launch();
    k_skip_grad<<<cdiv(P * 16, 256), 256, 0, s>>>(P * 16, N, N, 32, 16, n.gcat, n.gmid2, n.gbig);
    // c1b: out s1, in a1
    conv_dw<16, 16>(n, B, N, N, n.a1, n.gbig, n.s1, dwb(1).first, dwb(1).second, s);
    conv_fwd<16, 16>(B, N, N, n.gbig, n.s1, L[1].wb, nullptr, 0, n.gbig2, nullptr, s);     // grad a1
    // c1a: out a1, in x
    conv_dw<16, 16>(n, B, N, N, n.x, n.gbig2, n.a1, dwb(0).first, dwb(0).second, s);
    for (int k = 0; k < 9; k++) unpack(k);
}

void cnn_adam(Cnn &n, float lr, cudaStream_t s)
{
    n.step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)n.step), c2 = 1.0f - powf(b2, (float)n.step);
    note_launch();
    k_adam<<<cdiv((long)n.nparam, 256), 256, 0, s>>>((long)n.nparam, n.w, n.m, n.v, n.g, lr, b1, b2,
                                                    1e-8f, c1, c2);
    cnn_pack(n, s);
}

void cnn_output(Cnn &n, int B, int N, double h, double *p0, cudaStream_t s)
{
    const int N2 = N * N;
    const long P = (long)B * N2;
    note_launch();
    k_ysum_part<<<dim3(kRedBlocks, B), 256, 0, s>>>(N2, n.y32, n.rpart);
    note_launch();
    k_ymean_final<<<B, 256, 0, s>>>(N2, n.rpart, n.stats);
    note_launch();
    k_output<<<cdiv(P, 256), 256, 0, s>>>(P, N2, n.y32, n.stats, h * h * n.out_scale, p0);
}

// Inference with the inputs averaged over 2^levels x 2^levels blocks, the
// network run on the coarse grid (cell size h 2^levels) and its estimate
// interpolated back (bilinear, once per level); levels = 0 is plain
// inference.  N must be a multiple of 4 * 2^levels.
cudaError_t cnn_infer_levels(Cnn &n, int B, int N, double h, const double *rhs, const double *rho,
                             double *p0, int levels, cudaStream_t s)
{
    const int Nc = N >> levels;
    if (levels < 0 || levels > 6 || (Nc << levels) != N || Nc < 4 || Nc % 4) return cudaErrorInvalidValue;
    cudaError_t e = cnn_workspace(n, B, Nc);
    if (e != cudaSuccess) return e;
    if (levels == 0) {
        cnn_forward(n, B, N, h, rhs, rho, nullptr, s);
        cnn_output(n, B, N, h, p0, s);
        return cudaGetLastError();
    }
    // per level k = 1..levels: b_k, rho_k, p_k (B (N >> k)^2 each)
    size_t need = 0;
    for (int k = 1; k <= levels; k++) need += 3 * (size_t)B * (N >> k) * (N >> k);
    if (need > n.cbuf_cap) {
        if (n.cbuf) cudaFree(n.cbuf);
        n.cbuf = nullptr;
        n.cbuf_cap = 0;
        e = cudaMalloc(&n.cbuf, need * 8);
        if (e != cudaSuccess) return e;
        n.cbuf_cap = need;
    }
    double *bk[8], *rk[8], *pk[8];
    double *q = n.cbuf;
    for (int k = 1; k <= levels; k++) {
        const size_t m = (size_t)B * (N >> k) * (N >> k);
        bk[k] = q; rk[k] = q + m; pk[k] = q + 2 * m;
        q += 3 * m;
    }
    bk[0] = const_cast<double *>(rhs);
    rk[0] = const_cast<double *>(rho);
    pk[0] = p0;
    for (int k = 1; k <= levels; k++) {
        const long m = (long)B * (N >> k) * (N >> k);
        note_launch();
        k_restrict2<<<cdiv(m, 256), 256, 0, s>>>(m, N >> k, bk[k - 1], bk[k]);
        note_launch();
        k_restrict2<<<cdiv(m, 256), 256, 0, s>>>(m, N >> k, rk[k - 1], rk[k]);
    }
    const double hc = h * (double)(1 << levels);
    cnn_forward(n, B, Nc, hc, bk[levels], rk[levels], nullptr, s);
    cnn_output(n, B, Nc, hc, pk[levels], s);
    for (int k = levels; k >= 1; k--) {
        const long m = (long)B * (N >> (k - 1)) * (N >> (k - 1));
        note_launch();
        k_prolong2<<<cdiv(m, 256), 256, 0, s>>>(m, N >> k, pk[k], pk[k - 1]);
    }
    return cudaGetLastError();
}

// The network's pressure scale from training data: c = the median over the
// samples of rms(p - mean p) / (rms(b - mean b) h^2) (samples with b = const
// skipped; the mean of the two middle values for an even count).  Sets it
// and returns it in *c.
cudaError_t cnn_fit_scale(Cnn &n, int B, int N, double h, const double *rhs, const double *p,
                          double *c, cudaStream_t s)
{
    const int N2 = N * N;
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, (size_t)2 * B * 8);
    if (e != cudaSuccess) return e;
    note_launch(2);
    k_sample_rms<<<B, 256, 0, s>>>(N2, rhs, d);
    k_sample_rms<<<B, 256, 0, s>>>(N2, p, d + B);
    std::vector<double> hv((size_t)2 * B);
    e = cudaMemcpyAsync(hv.data(), d, (size_t)2 * B * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return e;
    std::vector<double> r;
    for (int k = 0; k < B; k++)
        if (hv[k] > 0.0) r.push_back(hv[B + k] / (hv[k] * h * h));
    if (r.empty()) return cudaErrorInvalidValue;
    std::sort(r.begin(), r.end());
    const size_t m = r.size();
    const double med = m % 2 ? r[m / 2] : 0.5 * (r[m / 2 - 1] + r[m / 2]);
    if (!(med > 0.0)) return cudaErrorInvalidValue;
    n.out_scale = med;
    *c = med;
    return cudaSuccess;
}

// Training: the pressure scale from all samples, then `steps` Adam steps on
// mini-batches of `batch` samples drawn with replacement by a SplitMix64
// stream of `seed`, the learning rate decaying tenfold over the run
// (lr0 0.1^(k / steps)); the batch losses land in losses_host (steps floats)
// with one synchronisation at the end.
cudaError_t cnn_train_loop(Cnn &n, int ns, int N, double h, const double *rhs, const double *rho,
                           const double *p, int steps, int batch, float lr0, unsigned long long seed,
                           float *losses_host, cudaStream_t s)
{
    double c = 0.0;
    cudaError_t e = cnn_fit_scale(n, ns, N, h, rhs, p, &c, s);
    if (e != cudaSuccess) return e;
    e = cnn_workspace(n, batch, N);
    if (e != cudaSuccess) return e;
    const long N2 = (long)N * N, nb = (long)batch * N2;
    std::vector<int> idx((size_t)steps * batch);
    unsigned long long st = seed;
    for (auto &v : idx) {
        st += 0x9E3779B97F4A7C15ULL;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        v = (int)((z ^ (z >> 31)) % (unsigned long long)ns);
    }
    char *mem = nullptr;
    const size_t bytes = al((size_t)nb * 8) * 3 + al(idx.size() * 4) + al((size_t)steps * 4);
    e = cudaMalloc(&mem, bytes);
    if (e != cudaSuccess) return e;
    double *gb = (double *)mem, *gr = (double *)(mem + al((size_t)nb * 8)),
           *gp = (double *)(mem + 2 * al((size_t)nb * 8));
    int *didx = (int *)(mem + 3 * al((size_t)nb * 8));
    float *dloss = (float *)(mem + 3 * al((size_t)nb * 8) + al(idx.size() * 4));
    e = cudaMemcpyAsync(didx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, s);
    for (int k = 0; k < steps && e == cudaSuccess; k++) {
        note_launch();
        k_gather3<<<cdiv(nb, 256), 256, 0, s>>>(nb, (int)N2, didx + (size_t)k * batch, rhs, rho, p,
                                                gb, gr, gp);
        cnn_forward(n, batch, N, h, gb, gr, gp, s);
        cnn_backward(n, batch, N, s);
        note_launch();
        k_loss_record<<<1, 32, 0, s>>>(batch, n.lsum, dloss + k);
        cnn_adam(n, (float)((double)lr0 * pow(0.1, (double)k / (double)steps)), s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(losses_host, dloss, (size_t)steps * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int f = 0;
    if (e == cudaSuccess) e = cnn_take_fault(&f);
    if (e == cudaSuccess && f) e = cudaErrorLaunchFailure;  // a tensor-core completion wait ran out
    cudaFree(mem);
    return e;
}

void cnn_set_scale(Cnn &n, double c) { n.out_scale = c; }
void cnn_set_tc(Cnn &n, int mode) { n.tc = mode; }

// Reads and clears the tensor-core convolutions' fault word.
cudaError_t cnn_take_fault(int *f)
{
    int z = 0;
    cudaError_t e = cudaMemcpyFromSymbol(f, g_cnn_fault, sizeof(int));
    if (e == cudaSuccess && *f) e = cudaMemcpyToSymbol(g_cnn_fault, &z, sizeof(int));
    return e;
}
const void *cnn_workspace_ptr(const Cnn &n) { return n.amem; }
const void *cnn_cbuf_ptr(const Cnn &n) { return n.cbuf; }
double cnn_get_scale(const Cnn &n) { return n.out_scale; }

size_t cnn_nparam(const Cnn &n) { return n.nparam; }
float *cnn_weights(Cnn &n) { return n.w; }
float *cnn_grads(Cnn &n) { return n.g; }
float *cnn_lsum(Cnn &n) { return n.lsum; }
int cnn_steps(const Cnn &n) { return n.step; }
void cnn_reset_adam(Cnn &n) { n.step = 0; cudaMemset(n.m, 0, n.nparam * 8); }

}  // namespace ibk
