// Stable LSD radix sort (8-bit digits) and exclusive scans.
//
// Used to order nodes (grain, Morton key), to canonicalise bond rows, and to
// bucket nodes by contact-grid cell.  Each pass: a per-tile digit histogram,
// one exclusive scan over the digit-major histogram, and a stable scatter in
// which every tile ranks its keys with warp match masks and per-warp digit
// counts, so equal keys keep their input order.
#include "pd_internal.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

template <typename K>
__global__ void k_radix_hist(const K *__restrict__ keys, int64_t n, int shift, int nblocks,
                             int64_t *__restrict__ hist)
{
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = base + r * RS_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(int)((keys[i] >> shift) & 0xFF)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

template <typename K>
__global__ void k_radix_scatter(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                K *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                                int shift, int nblocks, const int64_t *__restrict__ offs)
{
    __shared__ int64_t base_off[256];
    __shared__ int wcnt[RS_WARPS][256];
    __shared__ int run[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base_off[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
    run[tid] = 0;
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        for (int w = 0; w < RS_WARPS; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        int64_t i = base + r * RS_THREADS + tid;
        bool valid = i < n;
        K key = valid ? kin[i] : K(0);
        int d = valid ? (int)((key >> shift) & 0xFF) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {
            int s = run[tid];
            for (int w = 0; w < RS_WARPS; ++w) {
                int t = wcnt[w][tid];
                wcnt[w][tid] = s;
                s += t;
            }
            run[tid] = s;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = base_off[d] + wcnt[warp][d] + rank;
            kout[pos] = key;
            if (vin) vout[pos] = vin[i];
        }
        __syncthreads();
    }
}

// ---- scans ---------------------------------------------------------------
constexpr int SC_THREADS = 512;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t warp_sums[SC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < SC_THREADS / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SC_THREADS / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t prefix = (warp > 0 ? warp_sums[warp - 1] : 0) + x - v;
    if (total) *total = warp_sums[SC_THREADS / 32 - 1];
    __syncthreads();
    return prefix;
}

template <typename T>
__global__ void k_scan_reduce(const T *__restrict__ in, int64_t n, int64_t *__restrict__ sums)
{
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    int64_t s = 0;
    for (int r = 0; r < SC_ITEMS; ++r) {
        int64_t i = base + (int64_t)threadIdx.x * SC_ITEMS + r;
        if (i < n) s += (int64_t)in[i];
    }
    int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single-block exclusive scan of the block sums, in place; sums[m] = total
__global__ void k_scan_sums(int64_t *sums, int64_t m)
{
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < m; base += SC_THREADS) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < m ? sums[i] : 0;
        int64_t tot;
        int64_t p = block_exclusive_scan(v, &tot);
        if (i < m) sums[i] = carry + p;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[m] = carry;
}

template <typename T>
__global__ void k_scan_apply(const T *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                             const int64_t *__restrict__ sums, int64_t nb)
{
    int64_t base = (int64_t)blockIdx.x * SC_TILE;
    int64_t vals[SC_ITEMS];
    int64_t s = 0;
    for (int r = 0; r < SC_ITEMS; ++r) {
        int64_t i = base + (int64_t)threadIdx.x * SC_ITEMS + r;
        vals[r] = i < n ? (int64_t)in[i] : 0;
        s += vals[r];
    }
    int64_t p = block_exclusive_scan(s, nullptr) + sums[blockIdx.x];
    for (int r = 0; r < SC_ITEMS; ++r) {
        int64_t i = base + (int64_t)threadIdx.x * SC_ITEMS + r;
        if (i < n) out[i] = p;
        p += vals[r];
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = sums[nb];
}

template <typename T>
void scan_impl(const T *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st)
{
    int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    if (nb == 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), st);
        return;
    }
    k_scan_reduce<T><<<(unsigned)nb, SC_THREADS, 0, st>>>(in, n, tmp);
    k_scan_sums<<<1, SC_THREADS, 0, st>>>(tmp, nb);
    k_scan_apply<T><<<(unsigned)nb, SC_THREADS, 0, st>>>(in, out, n, tmp, nb);
}

template <typename K>
void radix_impl(K **k, K **kalt, uint32_t **v, uint32_t **valt, int64_t n, int bits, int64_t *hist,
                cudaStream_t st)
{
    if (n <= 1) return;
    int nb = radix_blocks(n);
    int64_t m = (int64_t)256 * nb;
    int64_t *offs = hist + m + 1;  // scan output after the histogram
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<K><<<nb, RS_THREADS, 0, st>>>(*k, n, shift, nb, hist);
        scan_impl<int64_t>(hist, offs, m, offs + m + 1, st);
        k_radix_scatter<K><<<nb, RS_THREADS, 0, st>>>(*k, v ? *v : nullptr, *kalt, v ? *valt : nullptr,
                                                      n, shift, nb, offs);
        K *t = *k; *k = *kalt; *kalt = t;
        if (v) { uint32_t *u = *v; *v = *valt; *valt = u; }
    }
}

}  // namespace

int radix_blocks(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

int64_t scan_tmp_size(int64_t n) { return (n + SC_TILE - 1) / SC_TILE + 2; }

int64_t radix_tmp_size(int64_t n)
{
    int64_t m = (int64_t)256 * radix_blocks(n);
    return 2 * (m + 1) + scan_tmp_size(m);
}

void radix_sort_u64(uint64_t **k, uint64_t **kalt, uint32_t **v, uint32_t **valt, int64_t n, int bits,
                    int64_t *hist, cudaStream_t st)
{
    radix_impl<uint64_t>(k, kalt, v, valt, n, bits, hist, st);
}

void radix_sort_u32(uint32_t **k, uint32_t **kalt, uint32_t **v, uint32_t **valt, int64_t n, int bits,
                    int64_t *hist, cudaStream_t st)
{
    radix_impl<uint32_t>(k, kalt, v, valt, n, bits, hist, st);
}

void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st)
{
    scan_impl<int64_t>(in, out, n, tmp, st);
}

void scan_exclusive_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp,
                               cudaStream_t st)
{
    scan_impl<int32_t>(in, out, n, tmp, st);
}
