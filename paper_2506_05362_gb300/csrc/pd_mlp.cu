// Bulk-stress surrogate: MLP with exact GELU, BF16 weights and activations,
// FP32 accumulation and FP32 master weights, MSE loss, Adam.
//
// GEMMs run on the tensor cores (mma.sync m16n8k16 BF16 -> FP32) with
// cp.async triple buffering and ldmatrix / ldmatrix.trans, so one kernel
// serves the three operand layouts of training:
//   forward      Z  = H  W^T + b      (A = H  row-major, B = W  row-major)
//   data grad    dH = dZ W            (A = dZ row-major, B = W  read transposed)
//   weight grad  dW = dZ^T H          (A = dZ read transposed, B = H read transposed)
// Epilogues fuse bias, GELU, the BF16 rounding of activations and GELU'.
// Weight gradients split the batch dimension across CTAs and reduce the FP32
// partials in a fixed order (bitwise reproducible).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "pd_internal.cuh"

typedef __nv_bfloat16 bf16;

namespace mlp {

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3, THREADS = 256;
constexpr int PAD = 8;  // bf16 elements of row padding in shared tiles

enum Epi : int {
    EPI_HIDDEN = 0,  // z = acc + b; Z (fp32, optional) and H = bf16(gelu(z))
    EPI_OUT = 1,     // y = acc + b, fp32, first n_valid columns
    EPI_DGELU = 2,   // dz = bf16(acc * gelu'(Zprev))
    EPI_PARTIAL = 3  // fp32 partial tile (split-K) to out + z * M * ldo
};

struct GemmArgs {
    int M, N, K;
    const bf16 *A;
    int lda;
    const bf16 *B;
    int ldb;
    int ksplit;           // rows of K per split (EPI_PARTIAL), else K
    const float *bias;
    bf16 *Zout;           // EPI_HIDDEN (nullable): pre-activations, stored as BF16
    bf16 *Hout;           // EPI_HIDDEN / EPI_DGELU
    const bf16 *Zin;      // EPI_DGELU
    float *out;           // EPI_OUT / EPI_PARTIAL
    int ldo;
    int n_valid;
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool pred)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    int sz = pred ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, const void *p)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(s));
}
__device__ __forceinline__ void mma_bf16(float *c, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared tile geometry: a non-transposed operand tile is [128 rows][BK] (K
// contiguous); a transposed one is [BK rows][128] (the M or N index contiguous).
template <bool T>
struct Tile {
    static constexpr int ROWS = T ? BK : BM;
    static constexpr int COLS = T ? BM : BK;
    static constexpr int LD = COLS + PAD;
    static constexpr int ELEMS = ROWS * LD;
};

// Loads the (row0, k0) tile of a row-major matrix X [R x C] (ld) into smem.
// Non-transposed: tile rows = R index (128), cols = C index (BK).
// Transposed:     tile rows = C index (BK), cols = R index (128); X is [K x R].
template <bool T>
__device__ __forceinline__ void load_tile(bf16 *s, const bf16 *X, int ld, int rows_total, int cols_total, int r0,
                                          int c0, int c_end)
{
    // 16-byte chunks: 8 bf16
    constexpr int CH_PER_ROW = Tile<T>::COLS / 8;
    constexpr int CHUNKS = Tile<T>::ROWS * CH_PER_ROW;
    for (int q = threadIdx.x; q < CHUNKS; q += THREADS) {
        const int r = q / CH_PER_ROW, cc = (q % CH_PER_ROW) * 8;
        int gr, gc;
        if (!T) { gr = r0 + r; gc = c0 + cc; } else { gr = c0 + r; gc = r0 + cc; }
        // non-transposed: gr over rows_total (M/N), gc over K (limit c_end)
        // transposed: gr over K rows (limit c_end), gc over M/N columns (rows_total)
        bool ok = !T ? (gr < rows_total && gc < c_end) : (gr < c_end && gc < rows_total);
        const bf16 *src = ok ? X + (size_t)gr * ld + gc : X;
        cp_async16(s + r * Tile<T>::LD + cc, src, ok);
    }
    (void)cols_total;
}

template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(THREADS) k_gemm(const GemmArgs g)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *sA = (bf16 *)smem_raw;
    bf16 *sB = sA + STAGES * Tile<AT>::ELEMS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, each 64 x 32
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = (EPI == EPI_PARTIAL) ? blockIdx.z * g.ksplit : 0;
    const int ke = (EPI == EPI_PARTIAL) ? min(g.K, kb + g.ksplit) : g.K;
    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const int nk = (ke - kb + BK - 1) / BK;
    // prologue
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nk) {
            load_tile<AT>(sA + s * Tile<AT>::ELEMS, g.A, g.lda, g.M, g.K, m0, kb + s * BK, ke);
            load_tile<BT>(sB + s * Tile<BT>::ELEMS, g.B, g.ldb, g.N, g.K, n0, kb + s * BK, ke);
        }
        cp_commit();
    }
    for (int it = 0; it < nk; ++it) {
        cp_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nx = it + STAGES - 1;
            if (nx < nk) {
                const int s = nx % STAGES;
                load_tile<AT>(sA + s * Tile<AT>::ELEMS, g.A, g.lda, g.M, g.K, m0, kb + nx * BK, ke);
                load_tile<BT>(sB + s * Tile<BT>::ELEMS, g.B, g.ldb, g.N, g.K, n0, kb + nx * BK, ke);
            }
            cp_commit();
        }
        const bf16 *a_s = sA + (it % STAGES) * Tile<AT>::ELEMS;
        const bf16 *b_s = sB + (it % STAGES) * Tile<BT>::ELEMS;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[4][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int rb = wm * 64 + mi * 16;
                if (!AT) {
                    const bf16 *p = a_s + (rb + (lane & 15)) * Tile<AT>::LD + kk + (lane >> 4) * 8;
                    ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], p);
                } else {
                    // matrices: (i0-7,r0-7), (i8-15,r0-7), (i0-7,r8-15), (i8-15,r8-15)
                    const int mat = lane >> 3, rr = lane & 7;
                    const int r = kk + rr + ((mat >> 1) << 3);
                    const int i = rb + ((mat & 1) << 3);
                    ldsm_x4_t(af[mi][0], af[mi][1], af[mi][2], af[mi][3], a_s + r * Tile<AT>::LD + i);
                }
            }
#pragma unroll
            for (int nj = 0; nj < 4; nj += 2) {
                const int cb = wn * 32 + nj * 8;
                unsigned r0, r1, r2, r3;
                if (!BT) {
                    // matrices: (j0-7,r0-7), (j0-7,r8-15), (j8-15,r0-7), (j8-15,r8-15)
                    const int mat = lane >> 3, rr = lane & 7;
                    const bf16 *p = b_s + (cb + rr + ((mat >> 1) << 3)) * Tile<BT>::LD + kk + ((mat & 1) << 3);
                    ldsm_x4(r0, r1, r2, r3, p);
                } else {
                    const int mat = lane >> 3, rr = lane & 7;
                    const int r = kk + rr + ((mat & 1) << 3);
                    const int j = cb + ((mat >> 1) << 3);
                    ldsm_x4_t(r0, r1, r2, r3, b_s + r * Tile<BT>::LD + j);
                }
                bfr[nj][0] = r0; bfr[nj][1] = r1; bfr[nj + 1][0] = r2; bfr[nj + 1][1] = r3;
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int nj = 0; nj < 4; ++nj)
                    mma_bf16(acc[mi][nj], af[mi][0], af[mi][1], af[mi][2], af[mi][3], bfr[nj][0], bfr[nj][1]);
        }
    }
    cp_wait<0>();
    // epilogue: thread (g = lane/4, t = lane%4) holds rows g, g+8 and cols 2t, 2t+1
    const int gr = lane >> 2, tc = (lane & 3) * 2;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm * 64 + mi * 16 + gr + h * 8;
                const int col = n0 + wn * 32 + nj * 8 + tc;
                if (row >= g.M) continue;
                const float v0 = acc[mi][nj][2 * h], v1 = acc[mi][nj][2 * h + 1];
                if (EPI == EPI_HIDDEN) {
                    if (col + 1 < g.N + 1 && col < g.N) {
                        const float z0 = v0 + g.bias[col], z1 = (col + 1 < g.N) ? v1 + g.bias[col + 1] : 0.f;
                        if (g.Zout) {
                            g.Zout[(size_t)row * g.ldo + col] = __float2bfloat16_rn(z0);
                            if (col + 1 < g.N) g.Zout[(size_t)row * g.ldo + col + 1] = __float2bfloat16_rn(z1);
                        }
                        __nv_bfloat162 hv = __floats2bfloat162_rn(gelu(z0), gelu(z1));
                        if (col + 1 < g.N)
                            *(__nv_bfloat162 *)(g.Hout + (size_t)row * g.ldo + col) = hv;
                        else
                            g.Hout[(size_t)row * g.ldo + col] = hv.x;
                    }
                } else if (EPI == EPI_OUT) {
                    if (col < g.n_valid) g.out[(size_t)row * g.ldo + col] = v0 + g.bias[col];
                    if (col + 1 < g.n_valid) g.out[(size_t)row * g.ldo + col + 1] = v1 + g.bias[col + 1];
                } else if (EPI == EPI_DGELU) {
                    if (col < g.N) {
                        const float d0 = v0 * gelu_grad(__bfloat162float(g.Zin[(size_t)row * g.ldo + col]));
                        const float d1 =
                            (col + 1 < g.N) ? v1 * gelu_grad(__bfloat162float(g.Zin[(size_t)row * g.ldo + col + 1])) : 0.f;
                        __nv_bfloat162 hv = __floats2bfloat162_rn(d0, d1);
                        if (col + 1 < g.N)
                            *(__nv_bfloat162 *)(g.Hout + (size_t)row * g.ldo + col) = hv;
                        else
                            g.Hout[(size_t)row * g.ldo + col] = hv.x;
                    }
                } else {
                    float *o = g.out + (size_t)blockIdx.z * g.M * g.ldo;
                    if (col < g.N) o[(size_t)row * g.ldo + col] = v0;
                    if (col + 1 < g.N) o[(size_t)row * g.ldo + col + 1] = v1;
                }
            }
}

template <bool AT, bool BT, int EPI>
void gemm(const GemmArgs &g, int splits, cudaStream_t st)
{
    const size_t smem = (size_t)STAGES * (Tile<AT>::ELEMS + Tile<BT>::ELEMS) * sizeof(bf16);
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_gemm<AT, BT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, splits);
    k_gemm<AT, BT, EPI><<<grid, THREADS, smem, st>>>(g);
}

// ---- small kernels ---------------------------------------------------------
__global__ void k_to_bf16_pad(const float *__restrict__ X, int64_t rows, int cols, int ldo, bf16 *out)
{
    const int64_t total = rows * ldo;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / ldo;
        const int c = (int)(q % ldo);
        out[q] = __float2bfloat16_rn(c < cols ? X[r * cols + c] : 0.f);
    }
}

// dY = bf16(2 (Y - T) / (B * nout)), padded to ldo; per-block loss partials
__global__ void k_loss(const float *__restrict__ Y, const float *__restrict__ T, int64_t rows, int nout, int ldo,
                       bf16 *dY, float *partial, bf16 *dYT, int64_t ldT)
{
    __shared__ float s[256];
    float acc = 0.f;
    const float scale = 2.0f / (float)(rows * nout);
    const int64_t total = rows * ldo;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / ldo;
        const int c = (int)(q % ldo);
        float d = 0.f;
        if (c < nout) {
            d = Y[r * nout + c] - T[r * nout + c];
            acc += d * d;
        }
        dY[q] = __float2bfloat16_rn(d * scale);
        if (dYT) dYT[(int64_t)c * ldT + r] = dY[q];  // transposed copy for the weight gradient
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

// fixed-order tree over the block partials (one block of 256 threads)
__global__ void k_loss_final(const float *__restrict__ partial, int nb, int64_t count, float *loss)
{
    __shared__ double s[256];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 256) acc += partial[b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(s[0] / (double)count);
}

// row sums of dZ^T (bf16 [n x ld], first `rows` columns) into gb: the bias
// gradient from the transposed copy, with coalesced reads; fixed order
constexpr int RS_THREADS = 1024;  // one block per column; two blocks fit an SM, so the columns take one wave
__global__ void __launch_bounds__(RS_THREADS) k_rowsum(const bf16 *__restrict__ dZT, int64_t rows, int64_t ld,
                                                       int n_valid, float *gb)
{
    __shared__ float s[RS_THREADS];
    const int c = blockIdx.x;
    float acc = 0.f;
    const bf16 *r = dZT + (int64_t)c * ld;  // ld is a multiple of 8: rows start 16-byte aligned
    const int64_t r8 = rows / 8;
    // RS_BATCH 16-byte loads of a thread are issued before any is added (one block
    // per column leaves few loads in flight otherwise); the additions keep the
    // order of a plain strided loop
    constexpr int RS_BATCH = 8;
    for (int64_t q0 = threadIdx.x; q0 < r8; q0 += (int64_t)RS_BATCH * blockDim.x) {
        uint4 w[RS_BATCH];
#pragma unroll
        for (int b = 0; b < RS_BATCH; ++b) {
            const int64_t q = q0 + (int64_t)b * blockDim.x;
            w[b] = q < r8 ? *(const uint4 *)(r + 8 * q) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int b = 0; b < RS_BATCH; ++b) {
            if (q0 + (int64_t)b * blockDim.x >= r8) break;
            const __nv_bfloat162 *h = (const __nv_bfloat162 *)&w[b];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h[e]);
                acc += f.x + f.y;
            }
        }
    }
    for (int64_t q = 8 * r8 + threadIdx.x; q < rows; q += blockDim.x) acc += __bfloat162float(r[q]);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = RS_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && c < n_valid) gb[c] = s[0];
}

// fixed-order sum of split-K partials into the gradient vector; rows < n_valid,
// cols < k_valid.  A block takes 32 consecutive outputs at a time with RD_PARTS
// warps: warp p adds splits p, p + RD_PARTS, p + 2 RD_PARTS, ... in that order
// (each a 128-byte load of the 32 outputs, several in flight), then warp 0 adds
// the RD_PARTS sums in order.  Many loads in flight per output instead of one
// thread walking all splits.
constexpr int RD_PARTS = 8;
__global__ void __launch_bounds__(32 * RD_PARTS) k_reduce_dw(const float *__restrict__ part, int splits, int N, int K,
                                                             int n_valid, int k_valid, float *gW)
{
    __shared__ float s[RD_PARTS][33];
    const int lane = threadIdx.x & 31, pp = threadIdx.x >> 5;
    const int64_t total = (int64_t)n_valid * k_valid;
    const size_t zs = (size_t)N * K;
    for (int64_t q0 = (int64_t)blockIdx.x * 32; q0 < total; q0 += (int64_t)gridDim.x * 32) {
        const int64_t q = q0 + lane;
        float acc = 0.f;
        if (q < total) {
            const int r = (int)(q / k_valid), c = (int)(q % k_valid);
            const float *src = part + (size_t)r * K + c;
#pragma unroll 4
            for (int z = pp; z < splits; z += RD_PARTS) acc += src[(size_t)z * zs];
        }
        s[pp][lane] = acc;
        __syncthreads();
        if (pp == 0 && q < total) {
            float t = s[0][lane];
#pragma unroll
            for (int w = 1; w < RD_PARTS; ++w) t += s[w][lane];
            gW[q] = t;
        }
        __syncthreads();
    }
}

inline int rd_blocks(int64_t total) { return (int)std::min<int64_t>((total + 31) / 32, 8192); }

// column sums of dZ (bf16, [rows x ld]) into gb (first n_valid), fixed order
__global__ void k_colsum(const bf16 *__restrict__ dZ, int64_t rows, int ld, int n_valid, float *gb)
{
    __shared__ float s[256];
    const int c = blockIdx.x;
    float acc = 0.f;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) acc += __bfloat162float(dZ[r * ld + c]);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && c < n_valid) gb[c] = s[0];
}

__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    }
}

// masters (layout W [out x in] then b) -> padded bf16 W [out_pad x in_pad] and fp32 bias [out_pad]
__global__ void k_pack_layer(const float *__restrict__ W, const float *__restrict__ b, int out, int in, int out_pad,
                             int in_pad, bf16 *Wb, float *bp, bf16 *WT)
{
    const int64_t total = (int64_t)out_pad * in_pad;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / in_pad), c = (int)(q % in_pad);
        const bf16 w = __float2bfloat16_rn((r < out && c < in) ? W[(int64_t)r * in + c] : 0.f);
        Wb[q] = w;
        if (WT) WT[(int64_t)c * out_pad + r] = w;  // [in_pad x out_pad], for the data gradient on tcgen05
        if (c == 0) bp[r] = r < out ? b[r] : 0.f;
    }
}

}  // namespace mlp

// ==============================================================================
struct pd_mlp {
    int device = 0;
    cudaStream_t st = nullptr;
    std::string err;
    int L = 0;
    int dims[9], pad[9];
    std::vector<int64_t> woff, boff;  // offsets of W_l, b_l in the parameter vector
    int64_t nparams = 0;
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    int64_t t = 0;
    bf16 *Wb[8] = {nullptr};
    bf16 *WT[8] = {nullptr};  // W transposed (tcgen05 training)
    float *bias[8] = {nullptr};
    // activations (capacity in rows)
    int64_t cap = 0;
    bf16 *H[9] = {nullptr};   // H[0] input (padded), H[l+1] after layer l (hidden)
    bf16 *Z[8] = {nullptr};   // pre-activations of hidden layers (BF16: only GELU' reads them)
    bf16 *dZ[9] = {nullptr};  // gradient w.r.t. pre-activation of layer l (dZ[L-1] = dY)
    // tcgen05 training: HT[l] = layer l's input transposed [pad[l] x ldT], dZT[l] =
    // dZ[l] transposed [pad[l+1] x ldT]
    bf16 *HT[8] = {nullptr}, *dZT[8] = {nullptr};
    int64_t ldT = 0;
    int tc_train = -1;        // -1: untried; 1: tcgen05 training works here; 0: mma.sync
    float *Y = nullptr, *Xf = nullptr, *Tf = nullptr;
    float *part = nullptr;    // split-K partials
    int64_t part_cap = 0;
    float *lpart = nullptr, *dloss = nullptr;
    unsigned *tc_err = nullptr;  // error word of the tcgen05 forward
    int path = 0;                // 0: tcgen05 forward when the shapes allow; 1: mma.sync only
    std::vector<void *> owned;
};

int mlp_forward_tc(int L, const int *dims, const int *pad, void *const *W, const float *const *bias, const float *X,
                   int64_t rows, float *Y, unsigned *err, int device, cudaStream_t st);
int mlp_forward_train_tc(int L, const int *dims, const int *pad, void *const *W, const float *const *bias,
                         const float *X, int64_t rows, float *Y, void *const *Z, void *const *HT, int64_t ldT,
                         unsigned *err, int device, cudaStream_t st);
int mlp_dgelu_tc(const void *dZ, const void *WT, const void *z, int64_t rows, int N, int K, void *out, void *outT,
                 int64_t ldT, unsigned *err, int device, cudaStream_t st);
int mlp_dw_tc(const void *dZT, const void *HT, int64_t rows, int64_t ldT, int M, int N, float *part, int max_splits,
              unsigned *err, int device, cudaStream_t st);

namespace {

using namespace mlp;

pd_status mfail(pd_mlp *m, pd_status s, const std::string &msg)
{
    if (m) m->err = msg;
    return s;
}

#define MCK(call)                                                                                 \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            return mfail(m, PD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
        }                                                                                         \
    } while (0)

template <typename T>
pd_status malloc_(pd_mlp *m, T **p, int64_t count)
{
    void *q = nullptr;
    if (cudaMalloc(&q, sizeof(T) * (size_t)std::max<int64_t>(count, 1)) != cudaSuccess) {
        cudaGetLastError();
        return mfail(m, PD_ENOMEM, "cudaMalloc failed in the MLP");
    }
    m->owned.push_back(q);
    *p = (T *)q;
    return PD_OK;
}

void mfree(pd_mlp *m, void *p)
{
    if (!p) return;
    for (size_t q = 0; q < m->owned.size(); ++q)
        if (m->owned[q] == p) { m->owned.erase(m->owned.begin() + q); break; }
    cudaFree(p);
}

int grid1(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 8192));
}

uint64_t splitmix64(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

pd_status pack_all(pd_mlp *m)
{
    for (int l = 0; l < m->L; ++l) {
        k_pack_layer<<<grid1((int64_t)m->pad[l + 1] * m->pad[l]), 256, 0, m->st>>>(
            m->master + m->woff[l], m->master + m->boff[l], m->dims[l + 1], m->dims[l], m->pad[l + 1], m->pad[l],
            m->Wb[l], m->bias[l], m->WT[l]);
    }
    MCK(cudaGetLastError());
    return PD_OK;
}

pd_status ensure_cap(pd_mlp *m, int64_t rows, bool train)
{
    if (rows <= m->cap && (!train || m->Z[0] || m->L == 1)) return PD_OK;
    int64_t cap = std::max<int64_t>(rows, m->cap);
    for (int l = 0; l <= m->L; ++l) { mfree(m, m->H[l]); m->H[l] = nullptr; mfree(m, m->dZ[l]); m->dZ[l] = nullptr; }
    for (int l = 0; l < m->L; ++l) { mfree(m, m->HT[l]); m->HT[l] = nullptr; mfree(m, m->dZT[l]); m->dZT[l] = nullptr; }
    for (int l = 0; l < m->L; ++l) { mfree(m, m->Z[l]); m->Z[l] = nullptr; }
    mfree(m, m->Y); mfree(m, m->Xf); mfree(m, m->Tf); mfree(m, m->lpart);
    pd_status s;
    for (int l = 0; l < m->L; ++l)
        if ((s = malloc_(m, &m->H[l], cap * m->pad[l]))) return s;
    if (train) {
        for (int l = 0; l + 1 < m->L; ++l)
            if ((s = malloc_(m, &m->Z[l], cap * m->pad[l + 1]))) return s;
        for (int l = 0; l < m->L; ++l)
            if ((s = malloc_(m, &m->dZ[l], cap * m->pad[l + 1]))) return s;
        m->ldT = (cap + 7) / 8 * 8;  // transposed rows: 16-byte strides for TMA
        for (int l = 0; l < m->L; ++l)
            if ((s = malloc_(m, &m->HT[l], m->ldT * m->pad[l])) || (s = malloc_(m, &m->dZT[l], m->ldT * m->pad[l + 1])))
                return s;
    }
    if ((s = malloc_(m, &m->Y, cap * m->dims[m->L]))) return s;
    if ((s = malloc_(m, &m->Xf, cap * m->dims[0]))) return s;
    if ((s = malloc_(m, &m->Tf, cap * m->dims[m->L]))) return s;
    if ((s = malloc_(m, &m->lpart, 8192))) return s;
    m->cap = cap;
    return PD_OK;
}

pd_status forward_dev(pd_mlp *m, const float *X, int64_t rows, float *Y, bool keepZ)
{
    if (!keepZ && m->path != 1) {
        void *W[8];
        const float *b[8];
        for (int l = 0; l < m->L; ++l) { W[l] = m->Wb[l]; b[l] = m->bias[l]; }
        if (mlp_forward_tc(m->L, m->dims, m->pad, W, b, X, rows, Y, m->tc_err, m->device, m->st) == 0)
            return PD_OK;
        if (m->path == 2) return mfail(m, PD_EINVAL, "the tcgen05 forward cannot run this network or GPU");
    }
    k_to_bf16_pad<<<grid1(rows * m->pad[0]), 256, 0, m->st>>>(X, rows, m->dims[0], m->pad[0], m->H[0]);
    for (int l = 0; l < m->L; ++l) {
        GemmArgs g;
        memset(&g, 0, sizeof(g));
        g.M = (int)rows; g.N = m->pad[l + 1]; g.K = m->pad[l];
        g.A = m->H[l]; g.lda = m->pad[l];
        g.B = m->Wb[l]; g.ldb = m->pad[l];
        g.ksplit = g.K;
        g.bias = m->bias[l];
        g.ldo = m->pad[l + 1];
        if (l + 1 < m->L) {
            g.Zout = keepZ ? m->Z[l] : nullptr;
            g.Hout = m->H[l + 1];
            gemm<false, false, EPI_HIDDEN>(g, 1, m->st);
        } else {
            g.out = Y;
            g.ldo = m->dims[m->L];
            g.n_valid = m->dims[m->L];
            gemm<false, false, EPI_OUT>(g, 1, m->st);
        }
    }
    MCK(cudaGetLastError());
    return PD_OK;
}

pd_status ensure_part(pd_mlp *m, int64_t need)
{
    if (need <= m->part_cap) return PD_OK;
    mfree(m, m->part);
    m->part = nullptr;
    pd_status s = malloc_(m, &m->part, need);
    if (s) return s;
    m->part_cap = need;
    return PD_OK;
}

// The same gradient on the tcgen05 kernels: the fused forward stores Z and the
// transposed layer inputs; dW = dZ^T H and dZ_{l-1} = (dZ_l W_l) GELU'(Z_{l-1})
// are tcgen05 GEMMs with K-major operands.  Returns -1 (nothing enqueued that
// changes results) when the kernels cannot run this network.
int backward_tc(pd_mlp *m, const float *X, const float *T, int64_t rows, float *dloss)
{
    const int L = m->L, nout = m->dims[L];
    for (int l = 0; l + 1 < L; ++l)
        if (m->pad[l + 1] % 32 != 0) return -1;
    void *W[8], *HT[8];
    const float *b[8];
    void *Z[8];
    for (int l = 0; l < L; ++l) { W[l] = m->Wb[l]; b[l] = m->bias[l]; HT[l] = m->HT[l]; Z[l] = m->Z[l]; }
    if (mlp_forward_train_tc(L, m->dims, m->pad, W, b, X, rows, m->Y, Z, HT, m->ldT, m->tc_err, m->device, m->st))
        return -1;
    const int nb = std::min(grid1(rows * m->pad[L]), 8192);
    k_loss<<<nb, 256, 0, m->st>>>(m->Y, T, rows, nout, m->pad[L], m->dZ[L - 1], m->lpart, m->dZT[L - 1], m->ldT);
    k_loss_final<<<1, 256, 0, m->st>>>(m->lpart, nb, rows * nout, dloss);
    const int max_splits = 128;
    for (int l = L - 1; l >= 0; --l) {
        const int N = m->pad[l + 1], K = m->pad[l];
        if (ensure_part(m, (int64_t)max_splits * ((N + 127) / 128 * 128) * K)) return -2;
        const int splits = mlp_dw_tc(m->dZT[l], m->HT[l], rows, m->ldT, N, K, m->part, max_splits, m->tc_err,
                                     m->device, m->st);
        if (splits <= 0) return -2;
        k_reduce_dw<<<rd_blocks((int64_t)m->dims[l + 1] * m->dims[l]), 32 * RD_PARTS, 0, m->st>>>(
            m->part, splits, N, K, m->dims[l + 1], m->dims[l], m->grad + m->woff[l]);
        k_rowsum<<<m->dims[l + 1], RS_THREADS, 0, m->st>>>(m->dZT[l], rows, m->ldT, m->dims[l + 1], m->grad + m->boff[l]);
        if (l > 0 && mlp_dgelu_tc(m->dZ[l], m->WT[l], m->Z[l - 1], rows, K, N, m->dZ[l - 1], m->dZT[l - 1], m->ldT,
                                  m->tc_err, m->device, m->st))
            return -2;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// gradient of the MSE loss into m->grad (parameter layout); loss to dloss (device)
pd_status backward_dev(pd_mlp *m, const float *X, const float *T, int64_t rows, float *dloss)
{
    if (m->path != 1) {
        const int r = backward_tc(m, X, T, rows, dloss);
        if (r == 0) return PD_OK;
        if (r == -2) return mfail(m, PD_ECUDA, "tcgen05 training kernels failed to launch");
        if (m->path == 2) return mfail(m, PD_EINVAL, "the tcgen05 kernels cannot train this network or GPU");
    }
    pd_status s = forward_dev(m, X, rows, m->Y, true);
    if (s) return s;
    const int L = m->L, nout = m->dims[L];
    const int nb = std::min(grid1(rows * m->pad[L]), 8192);
    k_loss<<<nb, 256, 0, m->st>>>(m->Y, T, rows, nout, m->pad[L], m->dZ[L - 1], m->lpart, nullptr, 0);
    k_loss_final<<<1, 256, 0, m->st>>>(m->lpart, nb, rows * nout, dloss);
    for (int l = L - 1; l >= 0; --l) {
        const int N = m->pad[l + 1], K = m->pad[l];
        // weight gradient: dW = dZ^T H, batch split across CTAs
        int splits = (int)std::max<int64_t>(1, std::min<int64_t>(128, rows / 512));
        int64_t ks = ((rows + splits - 1) / splits + BK - 1) / BK * BK;
        splits = (int)((rows + ks - 1) / ks);
        int64_t need = (int64_t)splits * N * K;
        if (need > m->part_cap) {
            mfree(m, m->part);
            m->part = nullptr;
            if ((s = malloc_(m, &m->part, need))) return s;
            m->part_cap = need;
        }
        GemmArgs g;
        memset(&g, 0, sizeof(g));
        g.M = N; g.N = K; g.K = (int)rows;
        g.A = m->dZ[l]; g.lda = N;
        g.B = m->H[l]; g.ldb = K;
        g.ksplit = (int)ks;
        g.out = m->part; g.ldo = K;
        gemm<true, true, EPI_PARTIAL>(g, splits, m->st);
        k_reduce_dw<<<rd_blocks((int64_t)m->dims[l + 1] * m->dims[l]), 32 * RD_PARTS, 0, m->st>>>(
            m->part, splits, N, K, m->dims[l + 1], m->dims[l], m->grad + m->woff[l]);
        k_colsum<<<m->dims[l + 1], 256, 0, m->st>>>(m->dZ[l], rows, N, m->dims[l + 1], m->grad + m->boff[l]);
        if (l > 0) {
            // data gradient: dH = dZ W, then dZ_{l-1} = dH * gelu'(Z_{l-1})
            GemmArgs d;
            memset(&d, 0, sizeof(d));
            d.M = (int)rows; d.N = K; d.K = N;
            d.A = m->dZ[l]; d.lda = N;
            d.B = m->Wb[l]; d.ldb = K;
            d.ksplit = N;
            d.Zin = m->Z[l - 1];
            d.Hout = m->dZ[l - 1];
            d.ldo = K;
            gemm<false, true, EPI_DGELU>(d, 1, m->st);
        }
    }
    MCK(cudaGetLastError());
    return PD_OK;
}

}  // namespace

extern "C" {

pd_status pd_mlp_create(const int *dims, int nlayers, uint64_t seed, int device, void *stream, pd_mlp **out)
{
    if (!out || !dims || nlayers < 1 || nlayers > 8) return PD_EINVAL;
    *out = nullptr;
    for (int l = 0; l <= nlayers; ++l)
        if (dims[l] < 1 || dims[l] > 1024) return PD_EINVAL;
    pd_mlp *m = new pd_mlp();
    m->device = device;
    m->st = (cudaStream_t)stream;
    m->L = nlayers;
    for (int l = 0; l <= nlayers; ++l) {
        m->dims[l] = dims[l];
        m->pad[l] = (dims[l] + 15) / 16 * 16;
    }
    int64_t off = 0;
    for (int l = 0; l < nlayers; ++l) {
        m->woff.push_back(off);
        off += (int64_t)dims[l + 1] * dims[l];
        m->boff.push_back(off);
        off += dims[l + 1];
    }
    m->nparams = off;
    pd_status s = PD_OK;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); delete m; return PD_ECUDA; }
    if ((s = malloc_(m, &m->master, off)) || (s = malloc_(m, &m->m, off)) || (s = malloc_(m, &m->v, off)) ||
        (s = malloc_(m, &m->grad, off)) || (s = malloc_(m, &m->dloss, 4)) || (s = malloc_(m, &m->tc_err, 1))) {
        pd_mlp_destroy(m);
        return s;
    }
    for (int l = 0; l < nlayers; ++l) {
        if ((s = malloc_(m, &m->Wb[l], (int64_t)m->pad[l + 1] * m->pad[l])) ||
            (s = malloc_(m, &m->WT[l], (int64_t)m->pad[l + 1] * m->pad[l])) ||
            (s = malloc_(m, &m->bias[l], m->pad[l + 1]))) {
            pd_mlp_destroy(m);
            return s;
        }
    }
    if (cudaMemsetAsync(m->tc_err, 0, sizeof(unsigned), m->st) != cudaSuccess) {
        cudaGetLastError();
        pd_mlp_destroy(m);
        return PD_ECUDA;
    }
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, SplitMix64
    std::vector<float> h(off, 0.f);
    uint64_t st = seed;
    for (int l = 0; l < nlayers; ++l) {
        const double bound = 1.0 / sqrt((double)dims[l]);
        for (int64_t q = 0; q < (int64_t)dims[l + 1] * dims[l]; ++q) {
            double u01 = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
            h[m->woff[l] + q] = (float)((2.0 * u01 - 1.0) * bound);
        }
    }
    s = pd_mlp_set_params(m, h.data());
    if (s) { pd_mlp_destroy(m); return s; }
    *out = m;
    return PD_OK;
}

void pd_mlp_destroy(pd_mlp *m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->st);
    for (void *p : m->owned) cudaFree(p);
    delete m;
}

const char *pd_mlp_last_error(const pd_mlp *m) { return m ? m->err.c_str() : "null"; }

pd_status pd_mlp_num_params(pd_mlp *m, int64_t *count)
{
    if (!m || !count) return PD_EINVAL;
    *count = m->nparams;
    return PD_OK;
}

pd_status pd_mlp_set_params(pd_mlp *m, const float *w)
{
    if (!m || !w) return PD_EINVAL;
    MCK(cudaSetDevice(m->device));
    for (int64_t q = 0; q < m->nparams; ++q)
        if (!isfinite(w[q])) return mfail(m, PD_EINVAL, "non-finite parameter");
    MCK(cudaMemcpyAsync(m->master, w, sizeof(float) * m->nparams, cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemsetAsync(m->m, 0, sizeof(float) * m->nparams, m->st));
    MCK(cudaMemsetAsync(m->v, 0, sizeof(float) * m->nparams, m->st));
    m->t = 0;
    pd_status s = pack_all(m);
    if (s) return s;
    MCK(cudaStreamSynchronize(m->st));
    return PD_OK;
}

pd_status pd_mlp_get_params(pd_mlp *m, float *w)
{
    if (!m || !w) return PD_EINVAL;
    MCK(cudaSetDevice(m->device));
    MCK(cudaMemcpyAsync(w, m->master, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    return PD_OK;
}

pd_status pd_mlp_forward_device(pd_mlp *m, const float *X, int64_t batch, float *Y)
{
    if (!m || !X || !Y || batch < 1 || batch > 0x7fffffff) return PD_EINVAL;
    MCK(cudaSetDevice(m->device));
    pd_status s = ensure_cap(m, batch, false);
    if (s) return s;
    return forward_dev(m, X, batch, Y, false);
}

pd_status pd_mlp_forward(pd_mlp *m, const float *X, int64_t batch, float *Y)
{
    if (!m || !X || !Y || batch < 1 || batch > 0x7fffffff) return PD_EINVAL;
    MCK(cudaSetDevice(m->device));
    pd_status s = ensure_cap(m, batch, false);
    if (s) return s;
    MCK(cudaMemcpyAsync(m->Xf, X, sizeof(float) * batch * m->dims[0], cudaMemcpyHostToDevice, m->st));
    s = forward_dev(m, m->Xf, batch, m->Y, false);
    if (s) return s;
    MCK(cudaMemcpyAsync(Y, m->Y, sizeof(float) * batch * m->dims[m->L], cudaMemcpyDeviceToHost, m->st));
    unsigned e = 0;
    MCK(cudaMemcpyAsync(&e, m->tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    if (e) {
        cudaMemsetAsync(m->tc_err, 0, sizeof(unsigned), m->st);
        return mfail(m, PD_ETIMEOUT, "a bounded wait of the tensor-core forward gave up");
    }
    return PD_OK;
}

pd_status pd_mlp_set_forward_path(pd_mlp *m, int path)
{
    if (!m || path < 0 || path > 2) return PD_EINVAL;
    m->path = path;
    return PD_OK;
}

static pd_status grad_impl(pd_mlp *m, const float *Xd, const float *Td, int64_t batch)
{
    pd_status s = ensure_cap(m, batch, true);
    if (s) return s;
    return backward_dev(m, Xd, Td, batch, m->dloss);
}

pd_status pd_mlp_grad(pd_mlp *m, const float *X, const float *T, int64_t batch, float *grad, float *loss)
{
    if (!m || !X || !T || !grad || batch < 1 || batch > 0x7fffffff) return PD_EINVAL;
    MCK(cudaSetDevice(m->device));
    pd_status s = ensure_cap(m, batch, true);
    if (s) return s;
    MCK(cudaMemcpyAsync(m->Xf, X, sizeof(float) * batch * m->dims[0], cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemcpyAsync(m->Tf, T, sizeof(float) * batch * m->dims[m->L], cudaMemcpyHostToDevice, m->st));
    s = grad_impl(m, m->Xf, m->Tf, batch);
    if (s) return s;
    MCK(cudaMemcpyAsync(grad, m->grad, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, m->st));
    if (loss) MCK(cudaMemcpyAsync(loss, m->dloss, sizeof(float), cudaMemcpyDeviceToHost, m->st));
    MCK(cudaStreamSynchronize(m->st));
    return PD_OK;
}

static pd_status adam(pd_mlp *m, float lr)
{
    m->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - pow(0.9, (double)m->t)), c2 = (float)(1.0 - pow(0.999, (double)m->t));
    k_adam<<<grid1(m->nparams), 256, 0, m->st>>>(m->master, m->grad, m->m, m->v, m->nparams, lr, b1, b2, 1e-8f,
                                                 c1, c2);
    return pack_all(m);
}

pd_status pd_mlp_train_step_device(pd_mlp *m, const float *X, const float *T, int64_t batch, float lr, float *loss)
{
    if (!m || !X || !T || batch < 1 || batch > 0x7fffffff || !(lr > 0)) return PD_EINVAL;
    MCK(cudaSetDevice(m->device));
    pd_status s = grad_impl(m, X, T, batch);
    if (s) return s;
    if (loss) MCK(cudaMemcpyAsync(loss, m->dloss, sizeof(float), cudaMemcpyDeviceToDevice, m->st));
    return adam(m, lr);
}

pd_status pd_mlp_train_step(pd_mlp *m, const float *X, const float *T, int64_t batch, float lr, float *loss)
{
    if (!m || !X || !T || batch < 1 || batch > 0x7fffffff || !(lr > 0)) return PD_EINVAL;
    MCK(cudaSetDevice(m->device));
    pd_status s = ensure_cap(m, batch, true);
    if (s) return s;
    MCK(cudaMemcpyAsync(m->Xf, X, sizeof(float) * batch * m->dims[0], cudaMemcpyHostToDevice, m->st));
    MCK(cudaMemcpyAsync(m->Tf, T, sizeof(float) * batch * m->dims[m->L], cudaMemcpyHostToDevice, m->st));
    s = grad_impl(m, m->Xf, m->Tf, batch);
    if (s) return s;
    if (loss) MCK(cudaMemcpyAsync(loss, m->dloss, sizeof(float), cudaMemcpyDeviceToHost, m->st));
    s = adam(m, lr);
    if (s) return s;
    MCK(cudaStreamSynchronize(m->st));
    return PD_OK;
}

}  // extern "C"
