// Uniform hashed cell grid shared by the bond builder and the contact search.
//
// A node at p falls in the integer cell c = floor((p - lo) / cs) (FP64), clamped
// to +-2^20 cells per axis.  Cells hash into a power-of-two bucket table; nodes
// are radix-sorted by bucket (stable, so each bucket lists its nodes in
// ascending index order) and a query walks the 27 cells around a node, keeping
// only nodes whose own cell is the visited cell.  The exact distance predicate
// is applied by the caller, so hashing and clamping never change a result.
#pragma once

#include "pd_internal.cuh"

struct GridView {
    double lo[3];
    double cs;                    // cell size
    uint32_t mask;                // bucket table size - 1
    const uint32_t *start;        // bucket -> first sorted entry (0xffffffff = empty)
    const uint32_t *end;          // bucket -> one past last
    const uint32_t *node;         // sorted entries -> node index
    const uint64_t *cell;         // node -> packed cell coordinates
    const float4 *pf;             // node -> FP32 (p - lo), .w = max |component| (prefilter)
};

// Conservative FP32 distance test.  pf = fl32(p - lo) carries an error of at
// most 2^-24 |pf|_inf per component; a difference of two such points and its
// squared norm in FP32 stay within r + 1.04e-7 (m_i + m_j) + 1.5e-7 r of the
// exact distance r (m = max |component|).  The bound below is four times that.
__device__ __forceinline__ float pf_slack(float cut, const float4 &a, const float4 &b)
{
    return cut * 1e-6f + 4e-7f * (a.w + b.w);
}
__device__ __forceinline__ float pf_dist2(const float4 &a, const float4 &b)
{
    const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

__device__ __forceinline__ int grid_coord(double p, double lo, double cs)
{
    double q = floor(__ddiv_rn(__dsub_rn(p, lo), cs));
    q = fmin(fmax(q, -1048576.0), 1048575.0);
    return (int)q;
}

__device__ __forceinline__ uint64_t grid_pack(int cx, int cy, int cz)
{
    return ((uint64_t)((uint32_t)(cx + 1048576) & 0x1fffffu) << 42) |
           ((uint64_t)((uint32_t)(cy + 1048576) & 0x1fffffu) << 21) |
           (uint64_t)((uint32_t)(cz + 1048576) & 0x1fffffu);
}

__device__ __forceinline__ uint32_t grid_hash(int cx, int cy, int cz, uint32_t mask)
{
    return (((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^ ((uint32_t)cz * 83492791u)) & mask;
}

// Build step kernels (pd_grid.cu).
void grid_build(GridView &g, const dbl4 *x4, const dbl4 *u4, int64_t n, double cs, uint32_t nbuckets,
                uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, uint32_t *start,
                uint32_t *end, uint64_t *cell, int64_t *tmp, float4 *pf, cudaStream_t st);
