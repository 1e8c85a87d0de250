// Internal declarations of libpd (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pd.h"

#define PD_MAX_WALLS 6

// 32-byte aligned double quadruple: one 256-bit load on sm_100+ parts
typedef double4_32a dbl4;

// device error bits (latched in pd_ctx::d_err)
enum : unsigned {
    PDE_NONFINITE = 1u,
    PDE_WALL = 2u,
    PDE_CAPACITY = 4u,   // contact candidate list overflow
    PDE_SKIN = 8u,       // a node moved more than half the skin between rebuilds
    PDE_BARRIER = 16u    // a grid-wide barrier of the multi-step kernel timed out
};

// what the fused step kernel does after the force evaluation
enum StepMode : int {
    MODE_FORCES = 0,  // store F and a; no velocity/position change
    MODE_FULL = 1,    // finish this step's kick, next half-kick, drift (writes other buffer)
    MODE_FINAL = 2    // finish this step's kick only
};

struct WallSet {
    int nw;
    double n[PD_MAX_WALLS][3];
    double v[PD_MAX_WALLS][3];
};

// Mixed-path node records: three float4 slots per node, (x_hi, c V), (u_hi,
// packed x_lo.xy) and (u_lo, packed x_lo.z), in one of three layouts (all give the
// same bits):
//   PD_PLANES = 0: interleaved, one 48-byte record per node (slot s of node i at
//     [3 i + s]);
//   PD_PLANES = 1 (default): three planes of n float4 (slot s of node i at
//     [s n + i]), so that the lanes of a group gathering neighbours that are
//     consecutive in the node order read one contiguous run per slot;
//   PD_PLANES = 2: an x plane and a u plane holding each node's (u_hi, u_lo) as
//     one 32-byte aligned pair, so that a neighbour's u is one 256-bit load (x at
//     [i], u_hi at [u0 + 2 i], u_lo at [u0 + 2 i + 1], u0 = n rounded up to even).
#ifndef PD_PLANES
#define PD_PLANES 1
#endif
constexpr int RECX = PD_PLANES ? 1 : 3;                              // element stride of the x slots
constexpr int REC = PD_PLANES == 0 ? 3 : (PD_PLANES == 1 ? 1 : 2);  // element stride of the u slots
// float4 offsets of node 0's u_hi and u_lo slots from the record base, and the
// float4 count of one record buffer
__host__ __device__ inline int64_t rec_uh0(int64_t n)
{
    return PD_PLANES == 0 ? 1 : (PD_PLANES == 1 ? n : (n + 1) & ~(int64_t)1);
}
__host__ __device__ inline int64_t rec_ul0(int64_t n) { return PD_PLANES == 1 ? 2 * n : rec_uh0(n) + 1; }
__host__ __device__ inline int64_t rec_float4s(int64_t n) { return PD_PLANES == 2 ? rec_uh0(n) + 2 * n : 3 * n; }

// Everything the force/update kernels need, passed by value.
struct StepParams {
    int64_t n;
    const int64_t *rowptr;
    const int32_t *col;
    uint32_t *brk;                 // broken bit per directed slot
    // mixed path: x, u, v as double-float pairs (hi, lo), a in FP32
    // mixed-path node records (layout above): (x_hi, c V) with x relative to the
    // bounding-box centre (static; c V set at bond build), (u_hi, packed x_lo.xy),
    // (u_lo, packed x_lo.z).  Two buffers (current / next) for u.
    const float4 *xh4;             // x slots of the current buffer (index RECX*i)
    const float4 *xl4;             // (x_lo, 0), dense
    const float4 *uh_in, *ul_in;   // = xh4 + rec_uh0(n), xh4 + rec_ul0(n) (index REC*i)
    float4 *uh_out, *ul_out;       // next buffer's u slots (index REC*i)
    float4 *vh, *vl;               // v (in place)
    float4 *af;                    // a = (F + b)/rho, stored for the next drift
    float dt_hi, dt_lo, hdt_hi, hdt_lo, inv_rho_f, bf[3], Rc_f;
    // FP64 state
    const dbl4 *x4;             // (x, V)
    const dbl4 *u_in;           // u, current buffer
    dbl4 *u_out;                // u, next buffer
    dbl4 *v;                    // velocity (in place)
    dbl4 *acc;                  // acceleration (F + b)/rho, stored
    dbl4 *F_out;                // force density (MODE_FORCES), may be null
    const int32_t *grain;
    // contact candidates (CSR; each entry = (j, bond slot or -1))
    int contact;
    const int64_t *cand_ptr;
    const int2 *cand;
    // constants
    double c, s0, Kn, Rc, rho, dt;
    float cf, s0f;
    int break_mode;
    int mode;
    WallSet walls;
    double *wall_pos;              // nw*3, current wall points (device)
    double b[3];
    // per-block partials and the last-block reduction
    double *partials;              // gridDim.x * PART_STRIDE
    unsigned *counter;
    unsigned *vmax_bits;           // max |v|^2 of the step as FP32 bits (atomicMax)
    unsigned *err;
    double *react;                 // nw*3 final wall reactions
    double *impulse;               // nw*3 sum over steps of dt * react (not in MODE_FORCES)
    double beta_d;                 // normal contact damping (0 = none)
    int conic;                     // conic micromodulus c (delta - |xi|)
    double delta;                  // horizon
    float delta_f;
    void *cand_fd;                 // damping + friction force per candidate: float4 (mixed) / dbl4 (FP64)
    double mu;                     // stick-slip friction coefficient (0 = none)
    double dt_f;                   // time step of the friction's stick branch (0 = the Coulomb limit)
    int pair_diss;                 // pair damping or friction on: k_pair_damping fills cand_fd
    int wall_overlap;              // inclusion-exclusion over orthogonal walls
    int wall_extra;                // walls with friction or inclusion-exclusion: the WX kernels run
    const double *wall_n;          // nw*3 wall normals (device copy, read by the overlap terms)
    const double *gl;              // Gauss-Legendre nodes, then weights, on [0, 1] (PD_GL each)
    double *disp;                  // accumulated displacement bound since last rebuild
    double skin;
    int *stale;                    // set when 2*disp >= skin
    // shared-memory tiles (mixed path; tile_cap = 0 disables)
    int tile_cap, tile_rows, tile_slot_cap;
    int64_t ntiles;
    double centre[3];              // origin of the split x (bounding-box centre)
    const int64_t *tile_ptr;
    const int32_t *ulist;
    uint16_t *lcol;                // bit 15 = broken (kept in step with brk)
    int32_t *colf;                 // mixed path: col with bit 31 = broken (kept in step with brk)
    const uint16_t *lrow;
    // each bond once (mixed path): pass 1 evaluates the slots of row i whose
    // neighbour index exceeds i and leaves the partner's factor at the mirror slot
    int pairs;
    const int32_t *split;          // per row: first slot whose neighbour index exceeds the row's
    const int32_t *mir;            // per slot: the slot of the same bond in the neighbour's row
    float *tb;                     // per slot: factor of the force term, written by pass 1
    float4 *fup;                   // per row: pass 1's force from the row's own slots
};

#define PART_STRIDE 20  // 18 reaction components, max|v| (multi-step kernel), spare
#define PD_GL 32        // Gauss-Legendre points of the multi-wall overlap integrals

// Radix sort of (key, value) pairs, LSD 8-bit digits, stable.  bits = number of
// low key bits to sort.  Buffers are ping-ponged; the result is in (*k, *v)
// (pointers swapped as needed).  hist must hold radix_tmp_size(n) int64.
int radix_blocks(int64_t n);
int64_t radix_tmp_size(int64_t n);
void radix_sort_u64(uint64_t **k, uint64_t **kalt, uint32_t **v, uint32_t **valt, int64_t n, int bits,
                    int64_t *hist, cudaStream_t st);
void radix_sort_u32(uint32_t **k, uint32_t **kalt, uint32_t **v, uint32_t **valt, int64_t n, int bits,
                    int64_t *hist, cudaStream_t st);
// Fragments (pd_frag.cu): connected components over intact bonds.  label and
// is_label are in caller order; parent and minc are n-element scratch.
void fragments_device(const int64_t *rowptr, const int32_t *col, const uint32_t *brk, const int32_t *perm,
                      int64_t n, int32_t *parent, int32_t *minc, int32_t *label, int64_t *is_label, cudaStream_t st);
// Scratch of the fragment statistics: sort keys and node indices (n each, two
// buffers), segment starts (nfrag + 1), and radix/scan workspace
// (max(radix_tmp_size(n), scan_tmp_size(nfrag + 1))).
struct FragSortScratch {
    uint64_t *k1, *k2;
    uint32_t *v1, *v2;
    int64_t *start, *tmp;
};
void fragment_stats_device(const int64_t *rowptr, const uint32_t *brk, const int32_t *perm, const dbl4 *x4,
                           const int32_t *label, const int64_t *fidx, int64_t n, int64_t nfrag,
                           unsigned long long *size, double *volume, unsigned long long *slots,
                           unsigned long long *intact, double *damage, FragSortScratch &w, cudaStream_t st);

// Exclusive scan of n int64 values (in may equal out); out[n] receives the total.
// tmp must hold scan_tmp_size(n) int64.
int64_t scan_tmp_size(int64_t n);
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp, cudaStream_t st);
void scan_exclusive_i32_to_i64(const int32_t *in, int64_t *out, int64_t n, int64_t *tmp,
                               cudaStream_t st);

// Step kernels (pd_step.cu)
void launch_step(const StepParams &p, int lanes, int blocks, cudaStream_t st);
// several MODE_FULL steps in one cooperative launch (see k_persist)
int persist_blocks(int lanes, int device, bool mixed, bool wx);
cudaError_t launch_persist(const StepParams &pa, const StepParams &pb, int nsteps, int lanes, int blocks,
                           unsigned *bar, unsigned absent, cudaStream_t st);
void launch_drift(const StepParams &p, cudaStream_t st);
// double-float state <-> FP64 (mixed path)
// double-float pair arrays with an element stride (1 for dense, REC for records)
void materialize_df(const float4 *hi, const float4 *lo, int stride, int64_t n, dbl4 *out, cudaStream_t st);
void split_df(const dbl4 *in, const float4 *xl, int64_t n, float4 *hi, float4 *lo, int stride, cudaStream_t st);
void fill_record_x(const float4 *xh4, int64_t n, float cf, float4 *rec, cudaStream_t st);
int step_blocks(int lanes, int device, bool mixed, bool tiled, size_t tile_smem);
size_t tiled_smem(int tile_cap, int tile_rows, int slot_cap);

// Device memory handle with the caller's allocator.
struct pd_ctx;
void *pd_dev_alloc(pd_ctx *c, size_t bytes);
void pd_dev_free(pd_ctx *c, void *p);
