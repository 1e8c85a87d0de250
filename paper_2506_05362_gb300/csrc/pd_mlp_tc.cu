// Fused MLP forward on the 5th-generation tensor cores (tcgen05, sm_100+).
//
// One persistent CTA per SM works on 128-row tiles of the batch, two at a time
// (slots 0 and 1, each with its activation tile in shared memory and its own
// 256-column TMEM accumulator), so that the tensor cores compute one slot's
// layer while the epilogue warps finish the other's:
//   warp 0      TMA producer: streams each layer's weights W_l [N x K] (BF16,
//               K-major) in 64-column chunks into a 3-stage ring, 128-byte
//               swizzle, completion counted on mbarriers;
//   warp 1      MMA issuer: one elected thread issues tcgen05.mma (M = 128,
//               N = layer width, K = 16 per instruction) from the activation
//               tile A and the weight stage into a TMEM accumulator, and
//               tcgen05.commit's to release stages and to signal the epilogue;
//   warps 2-17  epilogue: tcgen05.ld the accumulator (four warps per TMEM lane
//               quarter = 32 rows, each taking a quarter of the columns), add the
//               bias, exact-erf GELU, round to BF16 and write the next layer's A
//               tile in the swizzled layout; the last layer writes FP32 outputs.
//               They also stage the input tile with coalesced reads.
// Every mbarrier wait is bounded; on timeout the kernel records an error word,
// stops issuing, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <string.h>

#include "pd_internal.cuh"

namespace tc {

constexpr int TILE_M = 128;
constexpr int KCHUNK = 64;                    // BF16 columns per 128-byte swizzle atom
constexpr int STAGES = 3;
constexpr int MAX_N = 256;
constexpr int MAX_K = 256;
constexpr int A_BYTES = TILE_M * MAX_K * 2;   // 64 KiB: 4 atoms of 128 rows x 128 B
constexpr int W_STAGE_BYTES = MAX_N * KCHUNK * 2;  // 32 KiB
constexpr int EPI_THREADS = 512;              // 16 epilogue warps, 4 per TMEM lane quarter
constexpr int THREADS = 64 + EPI_THREADS;
constexpr int MAX_LAYERS = 8;
constexpr unsigned long long WAIT_NS = 1000000000ull;  // a wait gives up after 1 s

struct Layer {
    int K;        // padded input width (multiple of 16)
    int N;        // padded output width (multiple of 16, <= 256)
    int kchunks;  // ceil(K / 64)
    const float *bias;  // N_pad floats
};

struct Params {
    int L;
    Layer layer[MAX_LAYERS];
    const float *X;   // [rows x in_cols] FP32
    int in_cols;
    float *Y;         // [rows x out_cols] FP32
    int out_cols;
    int64_t rows;
    unsigned *err;    // error word (1 = a wait timed out)
    // training forward (nullable otherwise): Z[l] pre-activations of hidden layer l
    // [rows x N_l] BF16 (only GELU' reads them); HT[l] layer l's input transposed
    // [K_l x ldT] BF16
    __nv_bfloat16 *Z[MAX_LAYERS];
    __nv_bfloat16 *HT[MAX_LAYERS];
    int64_t ldT;
};

// ---- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: false once WAIT_NS of wall time have passed without the phase
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 256; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > WAIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row groups
// 1024 bytes apart (SBO), Blackwell descriptor version 1, layout SWIZZLE_128B
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(1u) << 16;                    // LBO (unused for swizzled K-major)
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;  // SBO
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= (uint64_t)2 << 61;                       // SWIZZLE_128B
    return d;
}

// instruction descriptor: D = F32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// 16 accumulator columns of this thread's TMEM lane, issued without waiting:
// the registers hold the values only after tmem_wait16 on them
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

// waits for this thread's TMEM loads; the registers pass through the wait, so
// no use of the loaded values can be scheduled before it
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU of two values at once on packed FP32x2 instructions, same method as
// gelu() below (Abramowitz & Stegun eq. 7.1.26 for erf, odd extension):
//   x = |z|/sqrt2, t = 1/(1 + p x), e = erf(x) = 1 - t P(t) exp(-x^2),
//   GELU = z/2 (1 + sign(z) e); the Horner coefficients carry the minus sign so
//   that e is one fused multiply-add, and sign(z) e is e with z's sign bit
//   (e >= 0).  exp(-x^2) = 2^(-x^2 log2 e) on the hardware ex2.
__device__ __forceinline__ float2 gelu2(float2 z)
{
    const float2 c = make_float2(0.70710678118654752f, 0.70710678118654752f);
    float2 x = __fmul2_rn(z, c);
    x.x = fabsf(x.x);
    x.y = fabsf(x.y);
    const float2 d = __ffma2_rn(make_float2(0.3275911f, 0.3275911f), x, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
    float2 q = __ffma2_rn(t, make_float2(-1.061405429f, -1.061405429f), make_float2(1.453152027f, 1.453152027f));
    q = __ffma2_rn(t, q, make_float2(-1.421413741f, -1.421413741f));
    q = __ffma2_rn(t, q, make_float2(0.284496736f, 0.284496736f));
    q = __ffma2_rn(t, q, make_float2(-0.254829592f, -0.254829592f));
    q = __fmul2_rn(t, q);  // -t P(t)
    const float2 w = __fmul2_rn(x, __fmul2_rn(x, make_float2(-1.4426950408889634f, -1.4426950408889634f)));
    const float2 ex = make_float2(ex2_approx(w.x), ex2_approx(w.y));
    const float2 e = __ffma2_rn(q, ex, make_float2(1.0f, 1.0f));
    const float2 es = make_float2(__uint_as_float(__float_as_uint(e.x) | (__float_as_uint(z.x) & 0x80000000u)),
                                  __uint_as_float(__float_as_uint(e.y) | (__float_as_uint(z.y) & 0x80000000u)));
    const float2 hz = __fmul2_rn(z, make_float2(0.5f, 0.5f));
    return __ffma2_rn(hz, es, hz);
}

// two floats rounded to BF16 (nearest-even), packed low = a, high = b, in registers
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&t);
}

// GELU z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 with erf from the rational
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions,
// eq. 7.1.26: erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
// t = 1 / (1 + p x), x >= 0, |error| <= 1.5e-7; odd extension to x < 0.  The
// error is far below the BF16 rounding of the activations (2^-9 relative).
__device__ __forceinline__ float gelu(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    const float e = 1.0f - poly * __expf(-x * x);
    return 0.5f * z * (1.0f + copysignf(e, z));
}

// byte offset of element (m, k) of a 128-row K-major BF16 tile in the 128-byte
// swizzled layout: atoms of 64 columns (16 KiB), 8-row groups of 1024 bytes,
// 16-byte chunk index XOR-ed with the row within its group
__device__ __forceinline__ uint32_t sw128_offset(int m, int k)
{
    const int atom = k >> 6, c = (k & 63) >> 3, r = m & 7, g = m >> 3;
    return (uint32_t)(atom * (TILE_M * 128) + g * 1024 + r * 128 + ((c ^ r) << 4) + ((k & 7) << 1));
}

// bias + GELU + BF16 of the 16 accumulator columns [c, c + 16) of row m, written
// to the next layer's swizzled A tile: the arithmetic of the whole-chunk path,
// element for element (c is a multiple of 16, so the bias loads are aligned)
__device__ __forceinline__ void epi16(const float *bias, const uint32_t (&r)[16], int c, unsigned char *sA, int m)
{
    float bb[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 t4 = __ldg((const float4 *)(bias + c) + i);
        bb[4 * i] = t4.x; bb[4 * i + 1] = t4.y; bb[4 * i + 2] = t4.z; bb[4 * i + 3] = t4.w;
    }
#pragma unroll
    for (int c8 = 0; c8 < 16; c8 += 8) {
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const float2 zz = __fadd2_rn(make_float2(__uint_as_float(r[c8 + e]), __uint_as_float(r[c8 + e + 1])),
                                         make_float2(bb[c8 + e], bb[c8 + e + 1]));
            const float2 g2 = gelu2(zz);
            pk[e / 2] = pack_bf16x2(g2.x, g2.y);
        }
        *(uint4 *)(sA + sw128_offset(m, c + c8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

}  // namespace tc

namespace {

using namespace tc;

struct Maps {
    CUtensorMap m[MAX_LAYERS];
};

// The CTA's tiles are blockIdx.x + k * gridDim.x, k = 0, 1, ...; they go in
// pairs (slot 0 = even k, slot 1 = odd k), each slot with its own activation
// tile in shared memory and its own TMEM accumulator.  All three roles walk the
// same item sequence: for each pair, for each layer, slot 0 then slot 1 (an odd
// last tile has slot-0 items only).  The MMAs of one slot's item run while the
// epilogue warps finish the other slot's previous item.
__device__ __forceinline__ int64_t pair_tile(int64_t r, int b) { return blockIdx.x + (2 * r + b) * (int64_t)gridDim.x; }

// input tile -> BF16 swizzled A tile (zero beyond the input width and the batch);
// consecutive threads take consecutive 8-column chunks of a row (coalesced reads)
__device__ __forceinline__ void stage_input(const Params &P, int64_t t, unsigned char *sA, int et)
{
    const int cpr = P.layer[0].kchunks * KCHUNK / 8;
    for (int ci = et; ci < TILE_M * cpr; ci += EPI_THREADS) {
        const int mm = ci / cpr, k0 = (ci - mm * cpr) * 8;
        const int64_t rr = t * TILE_M + mm;
        float xv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = k0 + e;
            xv[e] = (rr < P.rows && k < P.in_cols) ? P.X[rr * P.in_cols + k] : 0.f;
        }
        const uint4 pk = make_uint4(pack_bf16x2(xv[0], xv[1]), pack_bf16x2(xv[2], xv[3]), pack_bf16x2(xv[4], xv[5]),
                                    pack_bf16x2(xv[6], xv[7]));
        *(uint4 *)(sA + sw128_offset(mm, k0)) = pk;
        if (P.HT[0] && rr < P.rows) {  // training: the input transposed, for the first weight gradient
            const __nv_bfloat16 *hb = (const __nv_bfloat16 *)&pk;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (k0 + e < P.layer[0].K) P.HT[0][(int64_t)(k0 + e) * P.ldT + rr] = hb[e];
        }
    }
}

__global__ void __launch_bounds__(THREADS, 1) k_mlp_fwd_tc(const __grid_constant__ Maps maps, const Params P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzle atoms
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sW = base + 2 * A_BYTES;                   // weight stages
    uint64_t *full = (uint64_t *)(sW + STAGES * W_STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;  // [2], per slot
    uint64_t *a_ready = acc_full + 2;     // [2], per slot
    uint64_t *done = a_ready + 2;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; ++q) {
            mbar_init(full + q, 1);
            mbar_init(empty + q, 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(acc_full + q, 1);
            mbar_init(a_ready + q, EPI_THREADS);
        }
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {  // TMEM: two accumulators of 256 columns x 128 lanes (FP32)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * MAX_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int64_t ntiles = (P.rows + TILE_M - 1) / TILE_M;
    const int64_t my = ntiles > (int64_t)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t rounds = (my + 1) / 2;

    if (warp == 0) {
        // ---------------- TMA producer: each item streams its layer's weights
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int last_ph[STAGES];
            for (int q = 0; q < STAGES; ++q) last_ph[q] = -1;
            for (int64_t r = 0; r < rounds && !s_abort; ++r)
                for (int l = 0; l < P.L && !s_abort; ++l)
                    for (int b = 0; b < 2 && 2 * r + b < my && !s_abort; ++b)
                        for (int kc = 0; kc < P.layer[l].kchunks; ++kc) {
                            if (!mbar_wait(empty + s, ph ^ 1)) { atomicOr(P.err, 1u); s_abort = 1; break; }
                            mbar_expect_tx(full + s, (uint32_t)(P.layer[l].N * KCHUNK * 2));
                            tma_load_2d(sW + s * W_STAGE_BYTES, &maps.m[l], full + s, kc * KCHUNK, 0);
                            last_ph[s] = (int)ph;
                            if (++s == STAGES) { s = 0; ph ^= 1; }
                        }
            // no copy may still be landing in shared memory when the CTA exits
            for (int q = 0; q < STAGES; ++q)
                if (last_ph[q] >= 0 && !mbar_wait(full + q, (uint32_t)last_ph[q])) atomicOr(P.err, 1u);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, aph[2] = {0u, 0u};
            for (int64_t r = 0; r < rounds && !s_abort; ++r)
                for (int l = 0; l < P.L && !s_abort; ++l)
                    for (int b = 0; b < 2 && 2 * r + b < my && !s_abort; ++b) {
                        if (!mbar_wait(a_ready + b, aph[b])) { atomicOr(P.err, 1u); s_abort = 1; break; }
                        aph[b] ^= 1;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t idesc = idesc_bf16(TILE_M, P.layer[l].N);
                        const uint32_t d = tmem + (uint32_t)(b * MAX_N);
                        const unsigned char *sA = base + b * A_BYTES;
                        for (int kc = 0; kc < P.layer[l].kchunks; ++kc) {
                            if (!mbar_wait(full + s, ph)) { atomicOr(P.err, 1u); s_abort = 1; break; }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t a0 = smem_u32(sA + kc * (TILE_M * 128));
                            const uint32_t b0 = smem_u32(sW + s * W_STAGE_BYTES);
#pragma unroll
                            for (int kk = 0; kk < KCHUNK / 16; ++kk)
                                mma_bf16(d, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                                         (kc | kk) != 0);
                            mma_commit(empty + s);  // stage free once these MMAs completed
                            if (++s == STAGES) { s = 0; ph ^= 1; }
                        }
                        mma_commit(acc_full + b);  // this slot's accumulator complete
                    }
            // every MMA issued by this thread has completed before TMEM is freed
            mma_commit(done);
            if (!mbar_wait(done, 0)) atomicOr(P.err, 1u);
        }
    } else {
        // ---------------- epilogue warps 2..17: a warp may only read the TMEM lane
        // quarter warp % 4, so four warps share each quarter (32 rows) and split
        // the layer's columns between them
        const int q = warp & 3;
        const int part = (warp - 2) >> 2;  // 0..3
        const int m = q * 32 + lane;       // row of the tile owned by this thread
        const int et = threadIdx.x - 64;
        uint32_t accph[2] = {0u, 0u};
        bool stopped = false;
        for (int b = 0; b < 2 && b < my; ++b) stage_input(P, pair_tile(0, b), base + b * A_BYTES, et);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        for (int b = 0; b < 2 && b < my; ++b) mbar_arrive(a_ready + b);
        for (int64_t r = 0; r < rounds && !stopped; ++r)
            for (int l = 0; l < P.L && !stopped; ++l)
                for (int b = 0; b < 2 && 2 * r + b < my; ++b) {
                    const Layer &Ly = P.layer[l];
                    unsigned char *sA = base + b * A_BYTES;
                    const int64_t row = pair_tile(r, b) * TILE_M + m;
                    // the decision to stop is warp-uniform, so that no lane is left
                    // waiting in a warp-collective instruction
                    __syncwarp();
                    const bool ok = mbar_wait(acc_full + b, accph[b]);
                    if (!ok) { atomicOr(P.err, 1u); s_abort = 1; }
                    accph[b] ^= 1;
                    if (__any_sync(0xffffffffu, !ok || s_abort)) { stopped = true; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const bool last = (l == P.L - 1);
                    const int hw = ((Ly.N / 4 + 31) / 32) * 32;  // columns per part, whole 32-column loads
                    const int cend = min(Ly.N, (part + 1) * hw);
                    const uint32_t tacc = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * MAX_N);
                    // inference on whole 32-column chunks: the TMEM load of the next
                    // 16 columns is in flight while the current 16 go through GELU
                    const bool piped = !last && (Ly.N % 32) == 0 && !P.Z[l];
                    if (piped && part * hw < cend) {
                        uint32_t ra[16], rb[16];
                        __syncwarp();  // tcgen05.ld is warp-collective
                        tmem_ld16_issue(tacc + (uint32_t)(part * hw), ra);
                        tmem_wait16(ra);
                        for (int c0 = part * hw; c0 < cend; c0 += 32) {  // bounds uniform in the warp
                            __syncwarp();
                            tmem_ld16_issue(tacc + (uint32_t)(c0 + 16), rb);
                            epi16(Ly.bias, ra, c0, sA, m);
                            tmem_wait16(rb);
                            const bool more = c0 + 32 < cend;
                            if (more) {
                                __syncwarp();
                                tmem_ld16_issue(tacc + (uint32_t)(c0 + 32), ra);
                            }
                            epi16(Ly.bias, rb, c0 + 16, sA, m);
                            if (more) tmem_wait16(ra);
                        }
                    }
                    for (int c0 = part * hw; c0 < cend && !piped; c0 += 32) {
                        float v[32];
                        __syncwarp();  // tcgen05.ld is warp-collective
                        tmem_ld32(tacc + (uint32_t)c0, v);
                        if (!last && c0 + 32 <= Ly.N) {
                            // a whole chunk: its 32 biases in 8 vector loads (the bias
                            // array is 128-byte aligned at every 32-column boundary)
                            float bb[32];
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const float4 t4 = __ldg((const float4 *)(Ly.bias + c0) + i);
                                bb[4 * i] = t4.x; bb[4 * i + 1] = t4.y; bb[4 * i + 2] = t4.z; bb[4 * i + 3] = t4.w;
                            }
#pragma unroll
                            for (int c8 = 0; c8 < 32; c8 += 8) {
                                uint32_t pk[4];
                                float zs[8];
#pragma unroll
                                for (int e = 0; e < 8; e += 2) {
                                    const float2 zz = __fadd2_rn(make_float2(v[c8 + e], v[c8 + e + 1]),
                                                                 make_float2(bb[c8 + e], bb[c8 + e + 1]));
                                    zs[e] = zz.x;
                                    zs[e + 1] = zz.y;
                                    const float2 g2 = gelu2(zz);
                                    pk[e / 2] = pack_bf16x2(g2.x, g2.y);
                                }
                                *(uint4 *)(sA + sw128_offset(m, c0 + c8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                                if (P.Z[l] && row < P.rows) {  // training: Z for GELU', H^T for dW
                                    *(uint4 *)(P.Z[l] + row * Ly.N + c0 + c8) =
                                        make_uint4(pack_bf16x2(zs[0], zs[1]), pack_bf16x2(zs[2], zs[3]),
                                                   pack_bf16x2(zs[4], zs[5]), pack_bf16x2(zs[6], zs[7]));
                                    const __nv_bfloat16 *hb = (const __nv_bfloat16 *)pk;
#pragma unroll
                                    for (int e = 0; e < 8; ++e)
                                        P.HT[l + 1][(int64_t)(c0 + c8 + e) * P.ldT + row] = hb[e];
                                }
                            }
                        } else if (!last) {
#pragma unroll
                            for (int c8 = 0; c8 < 32; c8 += 8) {
                                float g[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    const int c = c0 + c8 + e;  // columns past N feed zero weights: keep them finite
                                    g[e] = c < Ly.N ? gelu(v[c8 + e] + __ldg(Ly.bias + c)) : 0.f;
                                }
                                *(uint4 *)(sA + sw128_offset(m, c0 + c8)) =
                                    make_uint4(pack_bf16x2(g[0], g[1]), pack_bf16x2(g[2], g[3]),
                                               pack_bf16x2(g[4], g[5]), pack_bf16x2(g[6], g[7]));
                            }
                        } else if (row < P.rows) {
#pragma unroll
                            for (int e = 0; e < 32; ++e)  // static indices keep v in registers
                                if (c0 + e < P.out_cols) P.Y[row * P.out_cols + c0 + e] = v[e] + __ldg(Ly.bias + c0 + e);
                        }
                    }
                    if (!last) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        mbar_arrive(a_ready + b);
                    } else if (2 * (r + 1) + b < my) {
                        // this slot's next tile; the accumulator has been read, and
                        // its last MMAs (which read sA) have completed
                        stage_input(P, pair_tile(r + 1, b), sA, et);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        mbar_arrive(a_ready + b);
                    }
                }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    __syncwarp();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * MAX_N));
}

typedef CUresult (*encode_fn_t)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn_t encoder()
{
    static encode_fn_t fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (encode_fn_t)p;
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

// ---- generic GEMM for training: C[M x N] = A[M x K] * B[N x K]^T ---------------
// Both operands K-major and fed by TMA (same 128-byte swizzle as above); one
// 128-row tile of C per CTA and one split of K (blockIdx.y); N <= 256.
//   GEMM_DGELU:   d = acc * GELU'(z) -> BF16 out[m][n] (ld N) and outT[n][m] (ld ldT)
//   GEMM_PARTIAL: acc -> FP32 part[split][m][n] (split-K partial sums)
namespace {

constexpr int G_EPI = 256;  // 8 epilogue warps, 2 per TMEM lane quarter
constexpr int G_THREADS = 64 + G_EPI;
constexpr int G_A_STAGE = TILE_M * KCHUNK * 2;  // 16 KiB
enum { GEMM_DGELU = 0, GEMM_PARTIAL = 1 };

struct GemmP {
    int M, N, kchunks, kcs;   // kcs: K chunks per split
    int mode;
    int64_t m_valid;          // rows of C that exist
    const __nv_bfloat16 *z;   // DGELU: pre-activation [M x N], BF16
    __nv_bfloat16 *out, *outT;
    int64_t ldT;
    float *part;              // PARTIAL
    unsigned *err;
};

// GELU'(z) = Phi(z) + z phi(z); Phi from the same Abramowitz-Stegun erf as gelu2,
// and exp(-z^2/2) is the exp(-x^2) of that erf
__device__ __forceinline__ float gelu_grad(float z)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    const float t = rcp_approx(fmaf(0.3275911f, x, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    const float ex = ex2_approx(-1.4426950408889634f * x * x);
    const float e = 1.0f - poly * ex;
    return 0.5f * (1.0f + copysignf(e, z)) + z * ex * 0.3989422804014327f;
}

__global__ void __launch_bounds__(G_THREADS, 1) k_gemm_tc(const __grid_constant__ CUtensorMap ma,
                                                          const __grid_constant__ CUtensorMap mb, const GemmP P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA = base;                                  // STAGES x 16 KiB
    unsigned char *sB = base + STAGES * G_A_STAGE;             // STAGES x 32 KiB
    uint64_t *full = (uint64_t *)(sB + STAGES * W_STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *acc_full = empty + STAGES;
    uint64_t *done = acc_full + 1;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; ++q) {
            mbar_init(full + q, 1);
            mbar_init(empty + q, 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(done, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(MAX_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int m0 = blockIdx.x * TILE_M;
    const int kc0 = blockIdx.y * P.kcs, kc1 = min(P.kchunks, kc0 + P.kcs);

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int last_ph[STAGES];
            for (int q = 0; q < STAGES; ++q) last_ph[q] = -1;
            for (int kc = kc0; kc < kc1; ++kc) {
                if (!mbar_wait(empty + s, ph ^ 1)) { atomicOr(P.err, 1u); s_abort = 1; break; }
                mbar_expect_tx(full + s, (uint32_t)(G_A_STAGE + P.N * KCHUNK * 2));
                tma_load_2d(sA + s * G_A_STAGE, &ma, full + s, kc * KCHUNK, m0);
                tma_load_2d(sB + s * W_STAGE_BYTES, &mb, full + s, kc * KCHUNK, 0);
                last_ph[s] = (int)ph;
                if (++s == STAGES) { s = 0; ph ^= 1; }
            }
            for (int q = 0; q < STAGES; ++q)
                if (last_ph[q] >= 0 && !mbar_wait(full + q, (uint32_t)last_ph[q])) atomicOr(P.err, 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            const uint32_t idesc = idesc_bf16(TILE_M, P.N);
            for (int kc = kc0; kc < kc1 && !s_abort; ++kc) {
                if (!mbar_wait(full + s, ph)) { atomicOr(P.err, 1u); s_abort = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(sA + s * G_A_STAGE);
                const uint32_t b0 = smem_u32(sB + s * W_STAGE_BYTES);
#pragma unroll
                for (int kk = 0; kk < KCHUNK / 16; ++kk)
                    mma_bf16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc, (kc != kc0 || kk != 0));
                mma_commit(empty + s);
                if (++s == STAGES) { s = 0; ph ^= 1; }
            }
            mma_commit(acc_full);
            mma_commit(done);
            if (!mbar_wait(done, 0)) atomicOr(P.err, 1u);
        }
    } else {
        const int q = warp & 3;
        const int part = (warp - 2) >> 2;  // 0..1
        const int m = q * 32 + lane;
        const int64_t row = (int64_t)m0 + m;
        __syncwarp();
        const bool ok = mbar_wait(acc_full, 0);
        if (!ok) { atomicOr(P.err, 1u); s_abort = 1; }
        if (!__any_sync(0xffffffffu, !ok || s_abort)) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int hw = ((P.N / 2 + 31) / 32) * 32;
            const int cend = min(P.N, (part + 1) * hw);
            for (int c0 = part * hw; c0 < cend; c0 += 32) {
                float v[32];
                __syncwarp();
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (row >= P.m_valid) continue;
                if (P.mode == GEMM_PARTIAL) {
                    float *dst = P.part + ((int64_t)blockIdx.y * P.M + row) * P.N + c0;
#pragma unroll
                    for (int e = 0; e < 32; e += 4)
                        if (c0 + e < P.N) *(float4 *)(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                } else {
                    const __nv_bfloat16 *zr = P.z + row * P.N + c0;
#pragma unroll
                    for (int e = 0; e < 32; e += 8) {
                        if (c0 + e >= P.N) break;
                        const uint4 zw = *(const uint4 *)(zr + e);  // 8 BF16 pre-activations
                        const float2 z01 = __bfloat1622float2(*(const __nv_bfloat162 *)&zw.x);
                        const float2 z23 = __bfloat1622float2(*(const __nv_bfloat162 *)&zw.y);
                        const float2 z45 = __bfloat1622float2(*(const __nv_bfloat162 *)&zw.z);
                        const float2 z67 = __bfloat1622float2(*(const __nv_bfloat162 *)&zw.w);
                        const float d0 = v[e] * gelu_grad(z01.x), d1 = v[e + 1] * gelu_grad(z01.y);
                        const float d2 = v[e + 2] * gelu_grad(z23.x), d3 = v[e + 3] * gelu_grad(z23.y);
                        const float d4 = v[e + 4] * gelu_grad(z45.x), d5 = v[e + 5] * gelu_grad(z45.y);
                        const float d6 = v[e + 6] * gelu_grad(z67.x), d7 = v[e + 7] * gelu_grad(z67.y);
                        const uint4 pk = make_uint4(pack_bf16x2(d0, d1), pack_bf16x2(d2, d3), pack_bf16x2(d4, d5),
                                                    pack_bf16x2(d6, d7));
                        *(uint4 *)(P.out + row * P.N + c0 + e) = pk;
                        const __nv_bfloat16 *hb = (const __nv_bfloat16 *)&pk;
#pragma unroll
                        for (int w = 0; w < 8; ++w) P.outT[(int64_t)(c0 + e + w) * P.ldT + row] = hb[w];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    __syncwarp();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MAX_N));
}

// K-major BF16 tensor map: rows x cols (cols = K, contiguous), row stride ld elements
bool kmajor_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows)
{
    encode_fn_t enc = encoder();
    if (!enc || (ld * 2) % 16 != 0 || ((uintptr_t)ptr & 15u) || box_rows > 256) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)KCHUNK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t gemm_tc_smem() { return 1024 + STAGES * (G_A_STAGE + W_STAGE_BYTES) + 128; }

int gemm_tc(const GemmP &P0, const void *A, int64_t a_rows, int64_t a_cols, int64_t a_ld, const void *B,
            int64_t b_ld, int splits, int device, cudaStream_t st)
{
    GemmP P = P0;
    if (P.N < 16 || P.N > MAX_N || P.N % 16 || splits < 1) return -1;
    CUtensorMap ma, mb;
    if (!kmajor_map(&ma, A, a_rows, a_cols, a_ld, TILE_M) || !kmajor_map(&mb, B, P.N, a_cols, b_ld, P.N)) return -1;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gemm_tc_smem());
        configured = true;
    }
    const dim3 grid((unsigned)((P.M + TILE_M - 1) / TILE_M), (unsigned)splits);
    k_gemm_tc<<<grid, G_THREADS, gemm_tc_smem(), st>>>(ma, mb, P);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

// dZ_prev = (dZ * W) . GELU'(Z): A = dZ [rows x K] (ld K), B = W^T [N x K] (ld K),
// z = Z [rows x N]; writes out [rows x N] and outT [N x ldT].  N <= 256.
int mlp_dgelu_tc(const void *dZ, const void *WT, const void *z, int64_t rows, int N, int K, void *out, void *outT,
                 int64_t ldT, unsigned *err, int device, cudaStream_t st)
{
    GemmP P;
    memset(&P, 0, sizeof(P));
    P.M = (int)((rows + TILE_M - 1) / TILE_M) * TILE_M;
    P.N = N;
    P.kchunks = (K + KCHUNK - 1) / KCHUNK;
    P.kcs = P.kchunks;
    P.mode = GEMM_DGELU;
    P.m_valid = rows;
    P.z = (const __nv_bfloat16 *)z;
    P.out = (__nv_bfloat16 *)out;
    P.outT = (__nv_bfloat16 *)outT;
    P.ldT = ldT;
    P.err = err;
    return gemm_tc(P, dZ, rows, K, K, WT, K, 1, device, st);
}

// split-K partials of dW = dZ^T H: A = dZ^T [M x rows] (ld ldT), B = H^T [N x rows]
// (ld ldT); part [splits x M x N] FP32.  Returns the number of splits used
// (<= 0 on failure).
int mlp_dw_tc(const void *dZT, const void *HT, int64_t rows, int64_t ldT, int M, int N, float *part, int max_splits,
              unsigned *err, int device, cudaStream_t st)
{
    GemmP P;
    memset(&P, 0, sizeof(P));
    P.M = M;
    P.N = N;
    P.kchunks = (int)((rows + KCHUNK - 1) / KCHUNK);
    const int mt = (M + TILE_M - 1) / TILE_M;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int splits = std::max(1, std::min(max_splits, sms / std::max(1, mt)));
    P.kcs = (P.kchunks + splits - 1) / splits;
    splits = (P.kchunks + P.kcs - 1) / P.kcs;  // no empty split
    P.mode = GEMM_PARTIAL;
    P.m_valid = M;
    P.part = part;
    P.err = err;
    return gemm_tc(P, dZT, M, rows, ldT, HT, ldT, splits, device, st) == 0 ? splits : -1;
}

size_t mlp_tc_smem() { return 1024 + 2 * A_BYTES + STAGES * W_STAGE_BYTES + 256; }

// Forward of an MLP whose layers all fit the fused kernel (K, N <= 256).
// W[l]: padded BF16 weights [pad_out x pad_in] row-major; bias[l]: pad_out
// floats.  Returns 0 on success, -1 if the shape is unsupported or the tensor
// maps cannot be made (the caller then uses the mma.sync kernels).
// Training forward: the same kernel also stores Z[l] (BF16 [rows x pad[l+1]],
// hidden layers) and HT[l] (BF16 [pad[l] x ldT], every layer's input
// transposed).  Hidden widths must be multiples of 32.
int mlp_forward_train_tc(int L, const int *dims, const int *pad, void *const *W, const float *const *bias,
                         const float *X, int64_t rows, float *Y, void *const *Z, void *const *HT, int64_t ldT,
                         unsigned *err, int device, cudaStream_t st);

int mlp_forward_tc(int L, const int *dims, const int *pad, void *const *W, const float *const *bias, const float *X,
                   int64_t rows, float *Y, unsigned *err, int device, cudaStream_t st)
{
    return mlp_forward_train_tc(L, dims, pad, W, bias, X, rows, Y, nullptr, nullptr, 0, err, device, st);
}

int mlp_forward_train_tc(int L, const int *dims, const int *pad, void *const *W, const float *const *bias,
                         const float *X, int64_t rows, float *Y, void *const *Z, void *const *HT, int64_t ldT,
                         unsigned *err, int device, cudaStream_t st)
{
    if (L < 1 || L > MAX_LAYERS || rows < 1) return -1;
    for (int l = 0; l < L; ++l)
        if (pad[l] > MAX_K || pad[l + 1] > MAX_N || pad[l + 1] % 16 != 0) return -1;
    if (Z)
        for (int l = 0; l + 1 < L; ++l)
            if (pad[l + 1] % 32 != 0) return -1;
    int major = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    if (major < 10) return -1;
    encode_fn_t enc = encoder();
    if (!enc) return -1;
    Maps maps;
    memset(&maps, 0, sizeof(maps));
    Params P;
    memset(&P, 0, sizeof(P));
    P.L = L;
    for (int l = 0; l < L; ++l) {
        const cuuint64_t gdim[2] = {(cuuint64_t)pad[l], (cuuint64_t)pad[l + 1]};
        const cuuint64_t gstride[1] = {(cuuint64_t)pad[l] * 2};
        const cuuint32_t box[2] = {(cuuint32_t)KCHUNK, (cuuint32_t)pad[l + 1]};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&maps.m[l], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, W[l], gdim, gstride, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -1;
        P.layer[l].K = pad[l];
        P.layer[l].N = pad[l + 1];
        P.layer[l].kchunks = (pad[l] + KCHUNK - 1) / KCHUNK;
        P.layer[l].bias = bias[l];
    }
    P.X = X;
    P.in_cols = dims[0];
    P.Y = Y;
    P.out_cols = dims[L];
    P.rows = rows;
    P.err = err;
    if (Z) {
        for (int l = 0; l < L; ++l) {
            P.Z[l] = (l + 1 < L) ? (__nv_bfloat16 *)Z[l] : nullptr;
            P.HT[l] = (__nv_bfloat16 *)HT[l];
        }
        P.ldT = ldT;
    }
    const size_t smem = mlp_tc_smem();
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int64_t ntiles = (rows + TILE_M - 1) / TILE_M;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sms);
    k_mlp_fwd_tc<<<grid, THREADS, smem, st>>>(maps, P);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
