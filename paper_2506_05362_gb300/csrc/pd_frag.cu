// Fragments: connected components of the graph of nodes and intact bonds (the
// paper identifies particles that split off, Sec. 1, without an algorithm).
//
// Lock-free union-find over the internal (Morton) node order: parent[i] <= i
// always holds (a root is hooked under a smaller root with atomicCAS), so every
// find walks a strictly decreasing chain and ends; path halving only ever
// replaces a parent by one of its ancestors.  After a full compression pass the
// label of a fragment is the smallest caller index among its nodes, so the
// result does not depend on the order in which the unions ran.
#include "pd_internal.cuh"

namespace {

__device__ __forceinline__ int32_t rep(int32_t *parent, int32_t x)
{
    volatile int32_t *vp = parent;
    int32_t cur = vp[x];
    if (cur != x) {
        int32_t prev = x, next;
        while (cur > (next = vp[cur])) {
            vp[prev] = next;  // path halving: next is an ancestor of prev
            prev = cur;
            cur = next;
        }
    }
    return cur;
}

__device__ __forceinline__ void unite(int32_t *parent, int32_t a, int32_t b)
{
    int32_t ra = rep(parent, a), rb = rep(parent, b);
    while (ra != rb) {
        if (ra > rb) { const int32_t t = ra; ra = rb; rb = t; }
        const int32_t old = atomicCAS(parent + rb, rb, ra);  // hook the larger root
        if (old == rb) break;
        rb = rep(parent, old);  // rb was hooked meanwhile: continue from its root
        ra = rep(parent, ra);
    }
}

__global__ void k_frag_init(int32_t *parent, int32_t *minc, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        parent[i] = (int32_t)i;
        minc[i] = 0x7fffffff;
    }
}

// one warp per row; each intact bond (i, j) with j > i joins the two sets
__global__ void k_frag_union(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                             const uint32_t *__restrict__ brk, int64_t n, int32_t *parent)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) {
            const int32_t j = col[k];
            if (j <= i) continue;
            if ((brk[k >> 5] >> (k & 31)) & 1u) continue;
            unite(parent, (int32_t)i, j);
        }
    }
}

// full compression, then the smallest caller index of each root's set
__global__ void k_frag_compress(int32_t *parent, const int32_t *__restrict__ perm, int32_t *minc, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = rep(parent, (int32_t)i);
        parent[i] = r;
        atomicMin(minc + r, perm[i]);
    }
}

// caller-order label of every node, and a 1 where a node is its fragment's label
__global__ void k_frag_label(const int32_t *__restrict__ parent, const int32_t *__restrict__ perm,
                             const int32_t *__restrict__ minc, int64_t n, int32_t *label, int64_t *is_label)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = perm[i], l = minc[parent[i]];
        label[c] = l;
        is_label[c] = (l == c) ? 1 : 0;
    }
}

// per-fragment integer sums (exact whatever the order of the atomics); fidx[c] =
// fragment index of label c (exclusive scan of is_label).  Also the sort key of
// every node, fragment index then caller index, for the fixed-order volume sums.
__global__ void k_frag_stats(const int64_t *__restrict__ rowptr, const uint32_t *__restrict__ brk,
                             const int32_t *__restrict__ perm, const int32_t *__restrict__ label,
                             const int64_t *__restrict__ fidx, int64_t n, unsigned long long *size,
                             unsigned long long *slots, unsigned long long *intact, uint64_t *key, uint32_t *node)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = perm[i];
        const int64_t q = fidx[label[c]];
        const int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
        unsigned long long ok = 0;
        for (int64_t k = k0; k < k1; ++k) ok += ((brk[k >> 5] >> (k & 31)) & 1u) ? 0ull : 1ull;
        atomicAdd(size + q, 1ull);
        atomicAdd(slots + q, (unsigned long long)(k1 - k0));
        atomicAdd(intact + q, ok);
        key[i] = ((uint64_t)q << 31) | (uint64_t)(uint32_t)c;
        node[i] = (uint32_t)i;
    }
}

// Volume of each fragment, one warp per fragment over its nodes in caller order
// (the sorted keys): lanes stride the segment, then a fixed xor butterfly, so the
// FP64 sum is the same on every run.
__global__ void k_frag_volume(const uint32_t *__restrict__ node, const int64_t *__restrict__ start,
                              const dbl4 *__restrict__ x4, int64_t nfrag, double *volume)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = w0; q < nfrag; q += nw) {
        const int64_t a = start[q], b = start[q + 1];
        double s = 0.0;
        for (int64_t t = a + lane; t < b; t += 32) s += x4[node[t]].w;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) volume[q] = s;
    }
}

__global__ void k_frag_damage(const unsigned long long *__restrict__ slots, const unsigned long long *__restrict__ intact,
                              int64_t nfrag, double *damage)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nfrag; q += (int64_t)gridDim.x * blockDim.x)
        damage[q] = slots[q] ? 1.0 - (double)intact[q] / (double)slots[q] : 0.0;
}

int grid_for(int64_t n, int per)
{
    const int64_t b = (n + per - 1) / per;
    return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

}  // namespace

void fragments_device(const int64_t *rowptr, const int32_t *col, const uint32_t *brk, const int32_t *perm,
                      int64_t n, int32_t *parent, int32_t *minc, int32_t *label, int64_t *is_label, cudaStream_t st)
{
    k_frag_init<<<grid_for(n, 256), 256, 0, st>>>(parent, minc, n);
    k_frag_union<<<grid_for(n * 32, 256), 256, 0, st>>>(rowptr, col, brk, n, parent);
    k_frag_compress<<<grid_for(n, 256), 256, 0, st>>>(parent, perm, minc, n);
    k_frag_label<<<grid_for(n, 256), 256, 0, st>>>(parent, perm, minc, n, label, is_label);
}

void fragment_stats_device(const int64_t *rowptr, const uint32_t *brk, const int32_t *perm, const dbl4 *x4,
                           const int32_t *label, const int64_t *fidx, int64_t n, int64_t nfrag,
                           unsigned long long *size, double *volume, unsigned long long *slots,
                           unsigned long long *intact, double *damage, FragSortScratch &w, cudaStream_t st)
{
    cudaMemsetAsync(size, 0, sizeof(unsigned long long) * nfrag, st);
    cudaMemsetAsync(slots, 0, sizeof(unsigned long long) * nfrag, st);
    cudaMemsetAsync(intact, 0, sizeof(unsigned long long) * nfrag, st);
    k_frag_stats<<<grid_for(n, 256), 256, 0, st>>>(rowptr, brk, perm, label, fidx, n, size, slots, intact, w.k1,
                                                   w.v1);
    int qbits = 1;
    while (qbits < 32 && ((int64_t)1 << qbits) <= nfrag) ++qbits;
    uint64_t *k = w.k1, *ka = w.k2;
    uint32_t *v = w.v1, *va = w.v2;
    radix_sort_u64(&k, &ka, &v, &va, n, 31 + qbits, w.tmp, st);
    scan_exclusive_i64((const int64_t *)size, w.start, nfrag, w.tmp, st);
    k_frag_volume<<<grid_for(nfrag * 32, 256), 256, 0, st>>>(v, w.start, x4, nfrag, volume);
    k_frag_damage<<<grid_for(nfrag, 256), 256, 0, st>>>(slots, intact, nfrag, damage);
}
