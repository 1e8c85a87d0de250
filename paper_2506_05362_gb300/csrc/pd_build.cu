// Set-up and rebuild kernels: node ordering, cell grid, bond CSR, contact
// candidate lists, and the small per-node reductions (damage, critical step,
// contact pairs for output).
#include "pd_build.cuh"
#include "pd_df.cuh"
#include "pd_grid.cuh"

namespace {

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double sq3(double a, double b, double c)
{
    return dadd(dadd(dmul(a, a), dmul(b, b)), dmul(c, c));
}

// ---- node ordering ---------------------------------------------------------
__device__ __forceinline__ uint64_t spread21(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void k_morton(const double *__restrict__ x, int64_t n, double lx, double ly, double lz,
                         double sx, double sy, double sz, uint64_t *key, uint32_t *val)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t qx = (uint64_t)fmin(fmax(floor((x[3 * i] - lx) * sx), 0.0), 2097151.0);
        uint64_t qy = (uint64_t)fmin(fmax(floor((x[3 * i + 1] - ly) * sy), 0.0), 2097151.0);
        uint64_t qz = (uint64_t)fmin(fmax(floor((x[3 * i + 2] - lz) * sz), 0.0), 2097151.0);
        key[i] = spread21(qx) | (spread21(qy) << 1) | (spread21(qz) << 2);
        val[i] = (uint32_t)i;
    }
}

__global__ void k_grain_keys(const int32_t *__restrict__ grain, const uint32_t *__restrict__ order, int64_t n,
                             uint64_t *key)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        key[k] = (uint64_t)(uint32_t)grain[order[k]];
}

__global__ void k_gather_nodes(const uint32_t *__restrict__ perm, int64_t n, const double *__restrict__ x,
                               const double *__restrict__ vol, const int32_t *__restrict__ grain,
                               const double *__restrict__ v0, int32_t *perm_out, int32_t *inv, dbl4 *x4,
                               int32_t *grain_out, dbl4 *v, float4 *xh4, float4 *xl4, double cx, double cy,
                               double cz)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[k];
        perm_out[k] = (int32_t)i;
        inv[i] = (int32_t)k;
        dbl4 a;
        a.x = x[3 * i]; a.y = x[3 * i + 1]; a.z = x[3 * i + 2]; a.w = vol[i];
        x4[k] = a;
        grain_out[k] = grain[i];
        dbl4 vv;
        vv.x = v0 ? v0[3 * i] : 0.0; vv.y = v0 ? v0[3 * i + 1] : 0.0; vv.z = v0 ? v0[3 * i + 2] : 0.0; vv.w = 0.0;
        v[k] = vv;
        if (xh4) {
            // split of x relative to the bounding-box centre (xi is translation invariant)
            const double rx = a.x - cx, ry = a.y - cy, rz = a.z - cz;
            float4 h, l;
            h.x = __double2float_rn(rx); l.x = __double2float_rn(rx - (double)h.x);
            h.y = __double2float_rn(ry); l.y = __double2float_rn(ry - (double)h.y);
            h.z = __double2float_rn(rz); l.z = __double2float_rn(rz - (double)h.z);
            h.w = (float)a.w; l.w = 0.f;
            xh4[k] = h;
            xl4[k] = l;
        }
    }
}

// ---- grid --------------------------------------------------------------------
__global__ void k_cell_keys(const dbl4 *__restrict__ x4, const dbl4 *__restrict__ u4, int64_t n, double lx,
                            double ly, double lz, double cs, uint32_t mask, uint32_t *key, uint32_t *val,
                            uint64_t *cell, float4 *pf)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        dbl4 a = x4[i];
        double px = a.x, py = a.y, pz = a.z;
        if (u4) {
            dbl4 u = u4[i];
            px = dadd(px, u.x); py = dadd(py, u.y); pz = dadd(pz, u.z);
        }
        int cx = grid_coord(px, lx, cs), cy = grid_coord(py, ly, cs), cz = grid_coord(pz, lz, cs);
        cell[i] = grid_pack(cx, cy, cz);
        const float fx = (float)dsub(px, lx), fy = (float)dsub(py, ly), fz = (float)dsub(pz, lz);
        pf[i] = make_float4(fx, fy, fz, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
        key[i] = grid_hash(cx, cy, cz, mask);
        val[i] = (uint32_t)i;
    }
}

__global__ void k_bucket_ranges(const uint32_t *__restrict__ key, int64_t n, uint32_t *start, uint32_t *end)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t b = key[e];
        if (e == 0 || key[e - 1] != b) start[b] = (uint32_t)e;
        if (e == n - 1 || key[e + 1] != b) end[b] = (uint32_t)(e + 1);
    }
}

// ---- bonds -------------------------------------------------------------------
// Filter test with the endpoints in canonical order (smaller caller index first).
__device__ bool filter_drops(const double *x1, const double *x2, const FilterSet &f)
{
    for (int q = 0; q < f.nf; ++q) {
        const double *p = f.a[q];
        if (f.kind[q] == 1) {
            double dx = dsub(x2[0], x1[0]), dy = dsub(x2[1], x1[1]), dz = dsub(x2[2], x1[2]);
            double num = dadd(dadd(dadd(dmul(p[0], x1[0]), dmul(p[1], x1[1])), dmul(p[2], x1[2])), p[3]);
            double den = dadd(dadd(dmul(p[0], dx), dmul(p[1], dy)), dmul(p[2], dz));
            if (den != 0.0) {
                double t = __ddiv_rn(-num, den);
                if (t > 0.0 && t < 1.0) {
                    double r0 = dadd(x1[0], dmul(t, dx)), r1 = dadd(x1[1], dmul(t, dy)), r2 = dadd(x1[2], dmul(t, dz));
                    if (r0 >= p[4] && r0 <= p[7] && r1 >= p[5] && r1 <= p[8] && r2 >= p[6] && r2 <= p[9]) return true;
                }
            }
        } else if (f.kind[q] == 2) {
            double R2 = dmul(p[3], p[3]);
            double d1 = sq3(dsub(x1[0], p[0]), dsub(x1[1], p[1]), dsub(x1[2], p[2]));
            double d2 = sq3(dsub(x2[0], p[0]), dsub(x2[1], p[1]), dsub(x2[2], p[2]));
            if (d1 < R2 || d2 < R2) return true;
        }
    }
    return false;
}

// Visits the bond partners of node i; FILL = false counts them, FILL = true
// writes keys (row << sh) | j.
template <bool FILL>
__global__ void k_bonds(const dbl4 *__restrict__ x4, const int32_t *__restrict__ grain,
                        const int32_t *__restrict__ perm, int64_t n, GridView g, double delta2, FilterSet f,
                        int64_t *cnt, const int64_t *__restrict__ off, uint64_t *keys, int sh)
{
    const float deltaf = (float)sqrt(delta2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const dbl4 a = x4[i];
        const float4 pi = g.pf[i];
        const int gi = grain[i];
        const int32_t ci = perm[i];
        const uint64_t pc = g.cell[i];
        const int cx = (int)((pc >> 42) & 0x1fffff) - 1048576, cy = (int)((pc >> 21) & 0x1fffff) - 1048576,
                  cz = (int)(pc & 0x1fffff) - 1048576;
        int64_t k = 0;
        int64_t base = FILL ? off[i] : 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const uint64_t want = grid_pack(cx + dx, cy + dy, cz + dz);
                    const uint32_t b = grid_hash(cx + dx, cy + dy, cz + dz, g.mask);
                    const uint32_t s = g.start[b];
                    if (s == 0xffffffffu) continue;
                    const uint32_t e = g.end[b];
                    for (uint32_t t = s; t < e; ++t) {
                        const int32_t j = (int32_t)g.node[t];
                        if (j == i || g.cell[j] != want || grain[j] != gi) continue;
                        // FP32 decides pairs clearly inside or outside the horizon;
                        // the exact FP64 predicate decides the band between
                        const float4 pj = g.pf[j];
                        const float d2f = pf_dist2(pi, pj), sl = pf_slack(deltaf, pi, pj);
                        const float hi = deltaf + sl, lo = deltaf - sl;
                        if (!(d2f < hi * hi)) continue;
                        const dbl4 bj = x4[j];
                        if (!(d2f < lo * lo)) {
                            const double r2 = sq3(dsub(bj.x, a.x), dsub(bj.y, a.y), dsub(bj.z, a.z));
                            if (!(r2 < delta2)) continue;
                        }
                        if (f.nf) {
                            const double pa[3] = {a.x, a.y, a.z}, pb[3] = {bj.x, bj.y, bj.z};
                            const bool drop = (ci < perm[j]) ? filter_drops(pa, pb, f) : filter_drops(pb, pa, f);
                            if (drop) continue;
                        }
                        if (FILL) keys[base + k] = ((uint64_t)i << sh) | (uint64_t)j;
                        ++k;
                    }
                }
        if (!FILL) cnt[i] = k;
    }
}

__global__ void k_keys_to_col(const uint64_t *__restrict__ keys, int64_t B, uint64_t mask, int32_t *col)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < B; k += (int64_t)gridDim.x * blockDim.x)
        col[k] = (int32_t)(keys[k] & mask);
}

// ---- contact candidates ---------------------------------------------------------
// Slot of j in the ascending row i, or -1.
__device__ __forceinline__ int64_t find_slot(const int64_t *rowptr, const int32_t *col, int64_t i, int32_t j)
{
    int64_t lo = rowptr[i], hi = rowptr[i + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1; else hi = mid;
    }
    return (lo < rowptr[i + 1] && col[lo] == j) ? lo : -1;
}

template <bool FILL>
__global__ void k_cand(const dbl4 *__restrict__ x4, const dbl4 *__restrict__ u4, const int32_t *__restrict__ grain,
                       const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n, GridView g,
                       double cut2, int64_t *cnt, const int64_t *__restrict__ off, int2 *cand, int64_t cap,
                       unsigned *err, double *disp, int *stale)
{
    if (FILL && blockIdx.x == 0 && threadIdx.x == 0) {
        *disp = 0.0;
        *stale = 0;
        if (off[n] > cap) atomicOr(err, (unsigned)PDE_CAPACITY);
    }
    if (FILL && off[n] > cap) return;
    const float cutf = (float)sqrt(cut2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 pi = g.pf[i];
        const int gi = grain[i];
        const uint64_t pc = g.cell[i];
        const int cx = (int)((pc >> 42) & 0x1fffff) - 1048576, cy = (int)((pc >> 21) & 0x1fffff) - 1048576,
                  cz = (int)(pc & 0x1fffff) - 1048576;
        int64_t k = 0;
        const int64_t base = FILL ? off[i] : 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const uint64_t want = grid_pack(cx + dx, cy + dy, cz + dz);
                    const uint32_t b = grid_hash(cx + dx, cy + dy, cz + dz, g.mask);
                    const uint32_t s = g.start[b];
                    if (s == 0xffffffffu) continue;
                    const uint32_t e = g.end[b];
                    for (uint32_t t = s; t < e; ++t) {
                        const int32_t j = (int32_t)g.node[t];
                        if (j == i || g.cell[j] != want) continue;
                        // a superset of the pairs closer than cut: the step kernel
                        // applies the exact FP64 contact predicate
                        const float4 pj = g.pf[j];
                        const float lim = cutf + pf_slack(cutf, pi, pj);
                        if (!(pf_dist2(pi, pj) < lim * lim)) continue;
                        if (FILL) {
                            int2 c;
                            c.x = j;
                            c.y = (grain[j] == gi) ? (int)find_slot(rowptr, col, i, j) : -1;
                            cand[base + k] = c;
                        }
                        ++k;
                    }
                }
        if (!FILL) {
            cnt[i] = k;
        } else {
            // ascending partner index (insertion sort; rows hold few candidates), so
            // that the step kernels add contact terms in an order that does not
            // depend on the grid's bucket order
            int2 *row = cand + base;
            for (int64_t a = 1; a < k; ++a) {
                const int2 c = row[a];
                int64_t b = a - 1;
                while (b >= 0 && row[b].x > c.x) {
                    row[b + 1] = row[b];
                    --b;
                }
                row[b + 1] = c;
            }
        }
    }
}

// Exact contact pairs from the candidate lists at the current state (for output).
template <bool FILL>
__global__ void k_pairs(const dbl4 *__restrict__ x4, const dbl4 *__restrict__ u4, const int32_t *__restrict__ perm,
                        const uint32_t *__restrict__ brk, const int64_t *__restrict__ cp, const int2 *__restrict__ cand,
                        int64_t n, double R2, int64_t *cnt, const int64_t *__restrict__ off, int32_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const dbl4 a = x4[i], ua = u4[i];
        const double px = dadd(a.x, ua.x), py = dadd(a.y, ua.y), pz = dadd(a.z, ua.z);
        int64_t k = 0;
        for (int64_t q = cp[i]; q < cp[i + 1]; ++q) {
            const int2 c = cand[q];
            if (c.y >= 0 && !((brk[c.y >> 5] >> (c.y & 31)) & 1u)) continue;
            const dbl4 bj = x4[c.x], uj = u4[c.x];
            const double r2 = sq3(dsub(dadd(bj.x, uj.x), px), dsub(dadd(bj.y, uj.y), py), dsub(dadd(bj.z, uj.z), pz));
            if (!(r2 < R2)) continue;
            if (FILL) {
                out[2 * (off[i] + k)] = perm[i];
                out[2 * (off[i] + k) + 1] = perm[c.x];
            }
            ++k;
        }
        if (!FILL) cnt[i] = k;
    }
}

// ---- reductions ------------------------------------------------------------------
__global__ void k_damage(const int64_t *__restrict__ rowptr, const uint32_t *__restrict__ brk,
                         const int32_t *__restrict__ perm, int64_t n, double *phi_caller)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
        int64_t broken = 0;
        for (int64_t k = k0; k < k1; ++k) broken += (brk[k >> 5] >> (k & 31)) & 1u;
        const int64_t nb0 = k1 - k0;
        phi_caller[perm[i]] = nb0 ? 1.0 - (double)(nb0 - broken) / (double)nb0 : 0.0;
    }
}

__global__ void k_stable_dt(const dbl4 *__restrict__ x4, const int64_t *__restrict__ rowptr,
                            const int32_t *__restrict__ col, int64_t n, double c, double rho, double delta,
                            int conic, double *dt_out)
{
    __shared__ double s_min[256];
    double best = INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
        if (k1 == k0) continue;
        const dbl4 a = x4[i];
        double sum = 0.0;
        for (int64_t k = k0; k < k1; ++k) {
            const dbl4 b = x4[col[k]];
            const double L = sqrt(sq3(b.x - a.x, b.y - a.y, b.z - a.z));
            sum += b.w * (conic ? c * (delta - L) : c) / L;
        }
        best = fmin(best, sqrt(2.0 * rho / sum));
    }
    s_min[threadIdx.x] = best;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) dt_out[blockIdx.x] = s_min[0];
}

// ---- canonical (caller-order) bond numbering ------------------------------------
// keys (caller row << sh | caller col), values = internal slot
__global__ void k_canon_keys(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                             const int32_t *__restrict__ perm, int64_t n, int sh, uint64_t *keys, uint32_t *vals)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ri = (uint64_t)(uint32_t)perm[i] << sh;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            keys[k] = ri | (uint64_t)(uint32_t)perm[col[k]];
            vals[k] = (uint32_t)k;
        }
    }
}

__global__ void k_canon_invert(const uint32_t *__restrict__ vals, int64_t B, int32_t *kc_of)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < B; q += (int64_t)gridDim.x * blockDim.x)
        kc_of[vals[q]] = (int32_t)q;
}

__global__ void k_row_len_caller(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ inv, int64_t n,
                                 int64_t *len)
{
    for (int64_t ic = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ic < n; ic += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = inv[ic];
        len[ic] = rowptr[i + 1] - rowptr[i];
    }
}

__global__ void k_col_caller(const int32_t *__restrict__ col, const int32_t *__restrict__ perm,
                             const int32_t *__restrict__ kc_of, int64_t B, int32_t *out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < B; k += (int64_t)gridDim.x * blockDim.x)
        out[kc_of[k]] = perm[col[k]];
}

__global__ void k_bits_to_bytes(const uint32_t *__restrict__ brk, const int32_t *__restrict__ kc_of, int64_t B,
                                uint8_t *out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < B; k += (int64_t)gridDim.x * blockDim.x)
        out[kc_of[k]] = (uint8_t)((brk[k >> 5] >> (k & 31)) & 1u);
}

// The internal bitset from one byte per canonical slot.  A warp builds one word
// at a time: lane l takes internal slot 32 w + l (coalesced reads of the slot
// map), and the word is the ballot of the lanes' bits.
__global__ void k_bytes_to_bits(const uint8_t *__restrict__ in, const int32_t *__restrict__ kc_of, int64_t B,
                                uint32_t *brk)
{
    const int64_t nw = (B + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += nwarps) {
        const int64_t k = (w << 5) + lane;
        const bool bit = k < B && in[kc_of[k]] != 0;
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) brk[w] = word;
    }
}

// Canonical packed bits (bit c % 32 of word c / 32 for canonical slot c) from the
// internal bitset: the words are cleared first, then every broken internal slot
// ORs its canonical bit (breaks are sparse, so the atomics are few).
__global__ void k_bits_to_packed(const uint32_t *__restrict__ brk, const int32_t *__restrict__ kc_of, int64_t B,
                                 uint32_t *out)
{
    const int64_t nw = (B + 31) >> 5;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = brk[w];
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const int64_t k = (w << 5) + b;
            if (k < B) {
                const int32_t c = kc_of[k];
                atomicOr(out + (c >> 5), 1u << (c & 31));
            }
        }
    }
}

// the internal bitset from canonical packed bits, a word per warp as above
__global__ void k_packed_to_bits(const uint32_t *__restrict__ in, const int32_t *__restrict__ kc_of, int64_t B,
                                 uint32_t *brk)
{
    const int64_t nw = (B + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += nwarps) {
        const int64_t k = (w << 5) + lane;
        bool bit = false;
        if (k < B) {
            const int32_t c = kc_of[k];
            bit = (in[c >> 5] >> (c & 31)) & 1u;
        }
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) brk[w] = word;
    }
}

// ---- shared-memory tiles -----------------------------------------------------------
// Tile t = rows [t*T, (t+1)*T).  Keys (t << sh | node) for every bond target and
// for every row itself; sorted and de-duplicated they give the tile's node list.
__global__ void k_tile_keys(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n, int T,
                            int sh, uint64_t *keys)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t t = (uint64_t)(i / T) << sh;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) keys[k] = t | (uint64_t)(uint32_t)col[k];
        keys[rowptr[n] + i] = t | (uint64_t)i;
    }
}

__global__ void k_unique_flags(const uint64_t *__restrict__ keys, int64_t m, int64_t *flag)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x)
        flag[q] = (q == 0 || keys[q] != keys[q - 1]) ? 1 : 0;
}

__global__ void k_unique_scatter(const uint64_t *__restrict__ keys, const int64_t *__restrict__ pos, int64_t m,
                                 int sh, int64_t ntiles, int32_t *ulist, int64_t *tile_ptr)
{
    const uint64_t mask = (1ull << sh) - 1ull;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[q];
        if (q == 0 || k != keys[q - 1]) ulist[pos[q]] = (int32_t)(k & mask);
        if (q == 0 || (k >> sh) != (keys[q - 1] >> sh)) tile_ptr[k >> sh] = pos[q];
        if (q == m - 1) tile_ptr[ntiles] = pos[m];
    }
}

__device__ __forceinline__ int32_t lsearch(const int32_t *__restrict__ a, int32_t len, int32_t v)
{
    int32_t lo = 0, hi = len;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// tile-local index of every bond target and of every row (tiles above cap get 0xffff)
__global__ void k_local_cols(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n, int T,
                             const int32_t *__restrict__ ulist, const int64_t *__restrict__ tile_ptr, int cap,
                             uint16_t *lcol, uint16_t *lrow)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / T;
        const int64_t base = tile_ptr[t];
        const int32_t len = (int32_t)(tile_ptr[t + 1] - base);
        const bool fits = len <= cap;
        lrow[i] = fits ? (uint16_t)lsearch(ulist + base, len, (int32_t)i) : 0xffffu;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            lcol[k] = fits ? (uint16_t)lsearch(ulist + base, len, col[k]) : 0xffffu;
    }
}

// broken flag of every slot copied into bit 15 of its local index
__global__ void k_sync_lcol_flags(const uint32_t *__restrict__ brk, int64_t B, uint16_t *lcol)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < B; k += (int64_t)gridDim.x * blockDim.x)
        lcol[k] = (uint16_t)((lcol[k] & 0x7fffu) | (((brk[k >> 5] >> (k & 31)) & 1u) << 15));
}

// neighbour index with the slot's broken flag in bit 31
__global__ void k_sync_colf_flags(const uint32_t *__restrict__ brk, const int32_t *__restrict__ col, int64_t B,
                                  int32_t *colf)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < B; k += (int64_t)gridDim.x * blockDim.x)
        colf[k] = (int32_t)((uint32_t)col[k] | (((brk[k >> 5] >> (k & 31)) & 1u) << 31));
}

// Index arrays of the each-bond-once passes: split[i] = first slot of row i whose
// neighbour index exceeds i (rows are sorted ascending); for each such slot k
// (bond i -> j), mir[k] = the slot of i in row j, and mir of that slot = k.  A
// bond without its reverse (the lists are symmetric by construction) sets *bad.
__global__ void k_pair_index(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n,
                             int32_t *split, int32_t *mir, unsigned *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
        int64_t a = k0, b = k1;  // first slot with col > i
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (col[m] > i) b = m; else a = m + 1;
        }
        split[i] = (int32_t)a;
        for (int64_t k = a; k < k1; ++k) {
            const int64_t j = col[k];
            int64_t lo = rowptr[j], hi = rowptr[j + 1];
            while (lo < hi) {
                const int64_t m = (lo + hi) >> 1;
                if (col[m] < i) lo = m + 1; else hi = m;
            }
            if (lo < rowptr[j + 1] && col[lo] == i) {
                mir[k] = (int32_t)lo;
                mir[lo] = (int32_t)k;
            } else {
                mir[k] = -1;
                atomicOr(bad, 1u);
            }
        }
    }
}

// ---- state conversion -----------------------------------------------------------
__global__ void k_to_caller(const dbl4 *__restrict__ in, const int32_t *__restrict__ perm, int64_t n, double *out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const dbl4 a = in[k];
        const int64_t i = perm[k];
        out[3 * i] = a.x; out[3 * i + 1] = a.y; out[3 * i + 2] = a.z;
    }
}

// flag |= bit when any of a[0..m) is not finite (one atomic per warp that saw one)
__global__ void k_nonfinite(const double *__restrict__ a, int64_t m, unsigned bit, unsigned *flag)
{
    bool bad = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(a[k]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, bit);
}

// flag |= bit when applying the caller-order doubles `staged` would change the
// current state: on the mixed path, when the split of a staged value (the one
// applying uses) differs from the live pair (hi, lo) at stride `stride`; else when
// it differs from the FP64 array d64.  The halves are compared as numbers (a zero
// of either sign counts as equal).  The live pairs lie on the FP64 grid, so a
// state read out and sent back unchanged splits into exactly the live pairs.
__global__ void k_state_differs(const double *__restrict__ staged, const int32_t *__restrict__ perm, int64_t n,
                                const float4 *__restrict__ hi, const float4 *__restrict__ lo, int stride,
                                const dbl4 *__restrict__ d64, unsigned bit, unsigned *flag)
{
    bool diff = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[k];
        const double a = staged[3 * i], b = staged[3 * i + 1], c = staged[3 * i + 2];
        if (hi) {
            const float4 h = hi[stride * k], l = lo[stride * k];
            const df sa = df_from_double(a), sb = df_from_double(b), sc = df_from_double(c);
            diff |= (sa.hi != h.x) | (sa.lo != l.x) | (sb.hi != h.y) | (sb.lo != l.y) | (sc.hi != h.z) |
                    (sc.lo != l.z);
        } else {
            const dbl4 q = d64[k];
            diff |= (a != q.x) | (b != q.y) | (c != q.z);
        }
    }
    if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) atomicOr(flag, bit);
}

__global__ void k_words_differ(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b, int64_t nw,
                               uint32_t last_mask, unsigned bit, unsigned *flag)
{
    bool diff = false;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x)
        diff |= ((a[w] ^ b[w]) & (w == nw - 1 ? last_mask : 0xffffffffu)) != 0u;
    if (__any_sync(0xffffffffu, diff) && (threadIdx.x & 31) == 0) atomicOr(flag, bit);
}

__global__ void k_from_caller(const double *__restrict__ in, const int32_t *__restrict__ perm, int64_t n, dbl4 *out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[k];
        dbl4 a;
        a.x = in[3 * i]; a.y = in[3 * i + 1]; a.z = in[3 * i + 2]; a.w = 0.0;
        out[k] = a;
    }
}

__global__ void k_split(const dbl4 *__restrict__ u, int64_t n, float4 *hi, float4 *lo)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const dbl4 a = u[k];
        float4 h, l;
        h.x = __double2float_rn(a.x); l.x = __double2float_rn(a.x - (double)h.x);
        h.y = __double2float_rn(a.y); l.y = __double2float_rn(a.y - (double)h.y);
        h.z = __double2float_rn(a.z); l.z = __double2float_rn(a.z - (double)h.z);
        h.w = 0.f; l.w = 0.f;
        hi[k] = h;
        lo[k] = l;
    }
}

__global__ void k_vmax(const dbl4 *__restrict__ v, int64_t n, double *out)
{
    __shared__ double s_m[256];
    double m = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const dbl4 a = v[k];
        m = fmax(m, a.x * a.x + a.y * a.y + a.z * a.z);
    }
    s_m[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_m[threadIdx.x] = fmax(s_m[threadIdx.x], s_m[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sqrt(s_m[0]);
}

}  // namespace

// ----------------------------------------------------------------------------------
static inline int grid_of(int64_t n, int threads = 256)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 8192) b = 8192;
    if (b < 1) b = 1;
    return (int)b;
}

void build_morton(const double *x_dev, int64_t n, const double lo[3], const double hi[3], uint64_t *key,
                  uint64_t *key_alt, uint32_t *val, uint32_t *val_alt, int grain_bits, const int32_t *grain_dev,
                  int64_t *tmp, uint32_t **order_out, cudaStream_t st)
{
    double s[3];
    for (int a = 0; a < 3; ++a) {
        double ext = hi[a] - lo[a];
        s[a] = ext > 0 ? 2097151.0 / ext : 0.0;
    }
    k_morton<<<grid_of(n), 256, 0, st>>>(x_dev, n, lo[0], lo[1], lo[2], s[0], s[1], s[2], key, val);
    uint64_t *k = key, *ka = key_alt;
    uint32_t *v = val, *va = val_alt;
    radix_sort_u64(&k, &ka, &v, &va, n, 63, tmp, st);
    if (grain_bits > 0) {
        k_grain_keys<<<grid_of(n), 256, 0, st>>>(grain_dev, v, n, k);
        radix_sort_u64(&k, &ka, &v, &va, n, grain_bits, tmp, st);
    }
    *order_out = v;
}

void gather_nodes(const uint32_t *order, int64_t n, const double *x, const double *vol, const int32_t *grain,
                  const double *v0, int32_t *perm, int32_t *inv, dbl4 *x4, int32_t *grain_out, dbl4 *v,
                  float4 *xh4, float4 *xl4, const double centre[3], cudaStream_t st)
{
    k_gather_nodes<<<grid_of(n), 256, 0, st>>>(order, n, x, vol, grain, v0, perm, inv, x4, grain_out, v, xh4, xl4,
                                               centre[0], centre[1], centre[2]);
}

void grid_build(GridView &g, const dbl4 *x4, const dbl4 *u4, int64_t n, double cs, uint32_t nbuckets,
                uint32_t *keys, uint32_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, uint32_t *start,
                uint32_t *end, uint64_t *cell, int64_t *tmp, float4 *pf, cudaStream_t st)
{
    g.cs = cs;
    g.mask = nbuckets - 1;
    k_cell_keys<<<grid_of(n), 256, 0, st>>>(x4, u4, n, g.lo[0], g.lo[1], g.lo[2], cs, g.mask, keys, vals, cell,
                                            pf);
    int bits = 0;
    while ((1u << bits) < nbuckets) ++bits;
    uint32_t *k = keys, *ka = keys_alt, *v = vals, *va = vals_alt;
    radix_sort_u32(&k, &ka, &v, &va, n, ((bits + 7) / 8) * 8, tmp, st);
    cudaMemsetAsync(start, 0xff, sizeof(uint32_t) * nbuckets, st);
    cudaMemsetAsync(end, 0, sizeof(uint32_t) * nbuckets, st);
    k_bucket_ranges<<<grid_of(n), 256, 0, st>>>(k, n, start, end);
    g.start = start;
    g.end = end;
    g.node = v;
    g.cell = cell;
    g.pf = pf;
}

void bonds_count(const dbl4 *x4, const int32_t *grain, const int32_t *perm, int64_t n, const GridView &g,
                 double delta, const FilterSet &f, int64_t *cnt, cudaStream_t st)
{
    k_bonds<false><<<grid_of(n, 128), 128, 0, st>>>(x4, grain, perm, n, g, delta * delta, f, cnt, nullptr, nullptr, 0);
}

void bonds_fill(const dbl4 *x4, const int32_t *grain, const int32_t *perm, int64_t n, const GridView &g,
                double delta, const FilterSet &f, const int64_t *off, uint64_t *keys, int sh, cudaStream_t st)
{
    k_bonds<true><<<grid_of(n, 128), 128, 0, st>>>(x4, grain, perm, n, g, delta * delta, f, nullptr, off, keys, sh);
}

void bonds_keys_to_col(const uint64_t *keys, int64_t B, int sh, int32_t *col, cudaStream_t st)
{
    k_keys_to_col<<<grid_of(B), 256, 0, st>>>(keys, B, (1ull << sh) - 1ull, col);
}

void cand_count(const dbl4 *x4, const dbl4 *u4, const int32_t *grain, const int64_t *rowptr, const int32_t *col,
                int64_t n, const GridView &g, double cut, int64_t *cnt, cudaStream_t st)
{
    k_cand<false><<<grid_of(n, 128), 128, 0, st>>>(x4, u4, grain, rowptr, col, n, g, cut * cut, cnt, nullptr,
                                                   nullptr, 0, nullptr, nullptr, nullptr);
}

void cand_fill(const dbl4 *x4, const dbl4 *u4, const int32_t *grain, const int64_t *rowptr, const int32_t *col,
               int64_t n, const GridView &g, double cut, const int64_t *off, int2 *cand, int64_t cap, unsigned *err,
               double *disp, int *stale, cudaStream_t st)
{
    k_cand<true><<<grid_of(n, 128), 128, 0, st>>>(x4, u4, grain, rowptr, col, n, g, cut * cut, nullptr, off, cand,
                                                  cap, err, disp, stale);
}

void pairs_count(const dbl4 *x4, const dbl4 *u4, const int32_t *perm, const uint32_t *brk, const int64_t *cp,
                 const int2 *cand, int64_t n, double Rc, int64_t *cnt, cudaStream_t st)
{
    k_pairs<false><<<grid_of(n), 256, 0, st>>>(x4, u4, perm, brk, cp, cand, n, Rc * Rc, cnt, nullptr, nullptr);
}

void pairs_fill(const dbl4 *x4, const dbl4 *u4, const int32_t *perm, const uint32_t *brk, const int64_t *cp,
                const int2 *cand, int64_t n, double Rc, const int64_t *off, int32_t *out, cudaStream_t st)
{
    k_pairs<true><<<grid_of(n), 256, 0, st>>>(x4, u4, perm, brk, cp, cand, n, Rc * Rc, nullptr, off, out);
}

void damage(const int64_t *rowptr, const uint32_t *brk, const int32_t *perm, int64_t n, double *phi,
            cudaStream_t st)
{
    k_damage<<<grid_of(n), 256, 0, st>>>(rowptr, brk, perm, n, phi);
}

int stable_dt_blocks(int64_t n) { return grid_of(n); }

void stable_dt(const dbl4 *x4, const int64_t *rowptr, const int32_t *col, int64_t n, double c, double rho,
               double delta, int conic, double *partial, cudaStream_t st)
{
    k_stable_dt<<<grid_of(n), 256, 0, st>>>(x4, rowptr, col, n, c, rho, delta, conic, partial);
}

void canon_keys(const int64_t *rowptr, const int32_t *col, const int32_t *perm, int64_t n, int sh, uint64_t *keys,
                uint32_t *vals, cudaStream_t st)
{
    k_canon_keys<<<grid_of(n, 128), 128, 0, st>>>(rowptr, col, perm, n, sh, keys, vals);
}

void canon_invert(const uint32_t *vals, int64_t B, int32_t *kc_of, cudaStream_t st)
{
    k_canon_invert<<<grid_of(B), 256, 0, st>>>(vals, B, kc_of);
}

void row_len_caller(const int64_t *rowptr, const int32_t *inv, int64_t n, int64_t *len, cudaStream_t st)
{
    k_row_len_caller<<<grid_of(n), 256, 0, st>>>(rowptr, inv, n, len);
}

void col_caller(const int32_t *col, const int32_t *perm, const int32_t *kc_of, int64_t B, int32_t *out,
                cudaStream_t st)
{
    k_col_caller<<<grid_of(B), 256, 0, st>>>(col, perm, kc_of, B, out);
}

void bits_to_bytes(const uint32_t *brk, const int32_t *kc_of, int64_t B, uint8_t *out, cudaStream_t st)
{
    k_bits_to_bytes<<<grid_of(B), 256, 0, st>>>(brk, kc_of, B, out);
}

void bytes_to_bits(const uint8_t *in, const int32_t *kc_of, int64_t B, uint32_t *brk, cudaStream_t st)
{
    k_bytes_to_bits<<<grid_of(B), 256, 0, st>>>(in, kc_of, B, brk);  // a warp per word
}

void bits_to_packed(const uint32_t *brk, const int32_t *kc_of, int64_t B, uint32_t *out, cudaStream_t st)
{
    const int64_t nw = (B + 31) / 32;
    cudaMemsetAsync(out, 0, sizeof(uint32_t) * (size_t)nw, st);
    k_bits_to_packed<<<grid_of(nw), 256, 0, st>>>(brk, kc_of, B, out);
}

void packed_to_bits(const uint32_t *in, const int32_t *kc_of, int64_t B, uint32_t *brk, cudaStream_t st)
{
    k_packed_to_bits<<<grid_of(B), 256, 0, st>>>(in, kc_of, B, brk);  // a warp per word
}

void to_caller(const dbl4 *in, const int32_t *perm, int64_t n, double *out, cudaStream_t st)
{
    k_to_caller<<<grid_of(n), 256, 0, st>>>(in, perm, n, out);
}

void check_finite(const double *a, int64_t m, unsigned bit, unsigned *flag, cudaStream_t st)
{
    k_nonfinite<<<grid_of(m), 256, 0, st>>>(a, m, bit, flag);
}

void state_differs(const double *staged, const int32_t *perm, int64_t n, const float4 *hi, const float4 *lo,
                   int stride, const dbl4 *d64, unsigned bit, unsigned *flag, cudaStream_t st)
{
    k_state_differs<<<grid_of(n), 256, 0, st>>>(staged, perm, n, hi, lo, stride, d64, bit, flag);
}

void words_differ(const uint32_t *a, const uint32_t *b, int64_t nw, uint32_t last_mask, unsigned bit, unsigned *flag,
                  cudaStream_t st)
{
    k_words_differ<<<grid_of(nw), 256, 0, st>>>(a, b, nw, last_mask, bit, flag);
}

void from_caller(const double *in, const int32_t *perm, int64_t n, dbl4 *out, cudaStream_t st)
{
    k_from_caller<<<grid_of(n), 256, 0, st>>>(in, perm, n, out);
}

void split_hilo(const dbl4 *u, int64_t n, float4 *hi, float4 *lo, cudaStream_t st)
{
    k_split<<<grid_of(n), 256, 0, st>>>(u, n, hi, lo);
}

int vmax_blocks(int64_t n)
{
    int b = grid_of(n);
    return b > 1024 ? 1024 : b;
}

void vmax(const dbl4 *v, int64_t n, double *partial, cudaStream_t st)
{
    k_vmax<<<vmax_blocks(n), 256, 0, st>>>(v, n, partial);
}

void build_tiles(const int64_t *rowptr, const int32_t *col, int64_t n, int64_t B, int T, int sh, int cap,
                 uint64_t *keys, uint64_t *keys_alt, int64_t *flag, int64_t *pos, int64_t *tmp, int32_t *ulist,
                 int64_t *tile_ptr, uint16_t *lcol, uint16_t *lrow, cudaStream_t st)
{
    const int64_t m = B + n;
    const int64_t ntiles = (n + T - 1) / T;
    int tbits = 1;
    while (((int64_t)1 << tbits) <= ntiles) ++tbits;
    k_tile_keys<<<grid_of(n, 128), 128, 0, st>>>(rowptr, col, n, T, sh, keys);
    uint64_t *k = keys, *ka = keys_alt;
    radix_sort_u64(&k, &ka, nullptr, nullptr, m, sh + tbits, tmp, st);
    k_unique_flags<<<grid_of(m), 256, 0, st>>>(k, m, flag);
    scan_exclusive_i64(flag, pos, m, tmp, st);
    k_unique_scatter<<<grid_of(m), 256, 0, st>>>(k, pos, m, sh, ntiles, ulist, tile_ptr);
    k_local_cols<<<grid_of(n, 128), 128, 0, st>>>(rowptr, col, n, T, ulist, tile_ptr, cap, lcol, lrow);
}

void sync_lcol_flags(const uint32_t *brk, int64_t B, uint16_t *lcol, cudaStream_t st)
{
    k_sync_lcol_flags<<<grid_of(B), 256, 0, st>>>(brk, B, lcol);
}

void pair_index(const int64_t *rowptr, const int32_t *col, int64_t n, int32_t *split, int32_t *mir, unsigned *bad,
                cudaStream_t st)
{
    k_pair_index<<<grid_of(n), 256, 0, st>>>(rowptr, col, n, split, mir, bad);
}

void sync_colf_flags(const uint32_t *brk, const int32_t *col, int64_t B, int32_t *colf, cudaStream_t st)
{
    if (B > 0) k_sync_colf_flags<<<grid_of(B), 256, 0, st>>>(brk, col, B, colf);
}
