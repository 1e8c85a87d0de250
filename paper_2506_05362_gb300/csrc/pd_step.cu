// Fused force evaluation and velocity-Verlet update.
//
// One launch per time step.  A group of G lanes owns one node i (row of the
// bond CSR) at a time, in a grid-stride loop over rows:
//   1. bond loop (Eq. peri-damage): each lane takes every G-th slot of row i,
//      skips broken slots (one bit per directed slot), computes the stretch,
//      breaks the bond (atomicOr of its bit) when s > s0, or accumulates
//      c s V_j (xi + eta)/|xi + eta|;
//   2. contact loop (Sec. 3.2, self-contact law): candidates of row i from the
//      skin list, exact |d|^2 < R_c^2 test in FP64, same-grain pairs skipped
//      while their bond bit is intact;
//   3. the group's partial sums are combined with xor shuffles;
//   4. the group leader adds the wall cap force (Sec. 4.1, FP64), forms
//      a = (F + b)/rho and performs the Verlet kick(s) and drift (Sec. 5.2).
// Positions are double-buffered: step n reads u^n and writes u^{n+1}, so every
// gather of step n sees the same state.  Per-block wall-reaction partials and
// the max |v| are combined by the last block to finish (fixed order, so runs
// are bitwise reproducible).
//
// Mixed path: u and x are held as float pairs (hi = RN(value), lo =
// RN(value - hi)); xi and eta are formed from hi and lo differences, which keeps
// the cancellation in u_j - u_i exact to ~2^-48 |u| while using FP32 units only.
// The stretch uses the cancellation-free form
//   s = eta . (2 xi + eta) / (|xi| (|xi + eta| + |xi|)),
// which equals (|xi + eta| - |xi|)/|xi| exactly in real arithmetic.
#include <cuda_bf16.h>

#include "pd_df.cuh"
#include "pd_internal.cuh"

namespace {

// A slot word of the bond stream: read once per step, so it is kept out of L1
// (no_allocate), where the gathered node records are reused.  1.5-3% per force
// evaluation against a plain read-only load (plate, hollow sphere, aggregate).
__device__ __forceinline__ int32_t ld_slot(const int32_t *a)
{
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(a));
    return v;
}

constexpr int STEP_THREADS = 256;
// bonds each lane keeps in flight per loop iteration, and the minimum resident
// blocks per SM the compiler must allow (register budget)
#ifndef PD_INFLIGHT
#define PD_INFLIGHT 3
#endif
// the global-gather mixed kernel: slot words loaded one batch ahead (software
// pipeline), PD_INFLIGHT_PF bonds per lane and batch
#ifndef PD_PREFETCH
#define PD_PREFETCH 1
#endif
#ifndef PD_INFLIGHT_PF
#define PD_INFLIGHT_PF 2
#endif
#ifndef PD_MINB_GLOBAL
#define PD_MINB_GLOBAL 4
#endif
#ifndef PD_MINB_TILED
#define PD_MINB_TILED 2
#endif

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

template <int G>
__device__ __forceinline__ float group_sum(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ double group_sum(double v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A step whose segment will be rolled back anyway: the contact list went stale in
// an earlier step (the mark is in *p.stale, or in the error word of an earlier
// kernel), or a rebuild overflowed the candidate list.  Every block reads values
// that only earlier kernels wrote (block 0 of k_step adds PDE_SKIN to the error
// word only when *p.stale is set), so all blocks of a launch agree and return
// together; the rest of the segment then costs little more than its launches.
__device__ __forceinline__ bool segment_doomed(const StepParams &p)
{
    return (p.contact && *(volatile const int *)p.stale) ||
           (*(volatile const unsigned *)p.err & (PDE_SKIN | PDE_CAPACITY));
}

// Wall cap force on a node at p (Sec. 4.1).  Returns error bits.
// ---- Several walls (Sec. 4.1.1) ------------------------------------------------
// In a frame whose axes point out through each wall, the part of the ball
// |r| < R beyond the planes X_k = t_k is W(t).  A negative threshold is turned
// into a positive one by the mirror image: {X > t} = ball - mirror{X > -t}, so
// W(t) is a signed sum (inclusion-exclusion over the negative thresholds) of
// the whole ball, caps, and corners whose thresholds are all >= 0.

// volume and first moments of {X > a, Y > b, Z > c} within |r| < R, a, b, c >= 0:
// the slice at height Z is the disk of radius s = sqrt(R^2 - Z^2) beyond the
// corner (a, b); its area Q and moments Qx, Qy are elementary, and the Z
// integral runs from c to Zm = sqrt(R^2 - a^2 - b^2) with Z = Zm - (Zm - c) u^2,
// which removes the square-root end point, by Gauss-Legendre in u.
__device__ __forceinline__ void corner_cut(const double *gl, double R, double a, double b, double c, double out[4])
{
    out[0] = out[1] = out[2] = out[3] = 0.0;
    const double R2 = R * R;
    if (a * a + b * b + c * c >= R2) return;
    const double Zm = sqrt(R2 - a * a - b * b), L = Zm - c;
#pragma unroll 1
    for (int q = 0; q < PD_GL; ++q) {
        const double u = gl[q], w = gl[PD_GL + q];
        const double Z = Zm - L * u * u;
        const double s2 = R2 - Z * Z;
        const double X1 = sqrt(fmax(s2 - b * b, 0.0)), Y1 = sqrt(fmax(s2 - a * a, 0.0));
        if (X1 <= a || Y1 <= b) continue;
        const double s = sqrt(s2);
        // Q = int_a^X1 (sqrt(s^2 - X^2) - b) dX, Qx = int X (...) dX, Qy by symmetry
        const double Q = 0.5 * (X1 * b + s2 * asin(fmin(X1 / s, 1.0))) - 0.5 * (a * Y1 + s2 * asin(a / s)) -
                         b * (X1 - a);
        const double Qx = (Y1 * Y1 * Y1 - b * b * b) / 3.0 - 0.5 * b * (X1 * X1 - a * a);
        const double Qy = (X1 * X1 * X1 - a * a * a) / 3.0 - 0.5 * a * (Y1 * Y1 - b * b);
        const double jw = 2.0 * L * u * w;
        out[0] += jw * Q;
        out[1] += jw * Qx;
        out[2] += jw * Qy;
        out[3] += jw * Z * Q;
    }
}

// W with thresholds t[k] >= 0 on the axes in `has` (bit k) and none on the others
__device__ void cut_term(const double *gl, double R, const double t[3], int has, double out[4])
{
    out[0] = out[1] = out[2] = out[3] = 0.0;
    const int m = __popc(has);
    if (m == 0) {
        out[0] = (4.0 * M_PI / 3.0) * R * R * R;
    } else if (m == 1) {
        const int k = __ffs(has) - 1;
        const double a = t[k];
        if (a >= R) return;
        out[0] = (M_PI / 3.0) * (R - a) * (R - a) * (2.0 * R + a);
        out[1 + k] = (M_PI / 4.0) * (R * R - a * a) * (R * R - a * a);
    } else if (m == 2) {
        const int k = __ffs(has) - 1, l = __ffs(has & ~(1 << k)) - 1;
        double c2[4];
        corner_cut(gl, R, t[k], t[l], 0.0, c2);  // half of the two-plane region (Z > 0)
        out[0] = 2.0 * c2[0];
        out[1 + k] = 2.0 * c2[1];
        out[1 + l] = 2.0 * c2[2];
    } else {
        corner_cut(gl, R, t[0], t[1], t[2], out);
    }
}

// W beyond the thresholds th[k] (any sign above -R) on the axes in `has`
__device__ void ball_cut(const double *gl, double R, const double th[3], int has, double out[4])
{
    int neg = 0;
    for (int k = 0; k < 3; ++k)
        if (((has >> k) & 1) && th[k] < 0.0) neg |= 1 << k;
    const double t[3] = {fabs(th[0]), fabs(th[1]), fabs(th[2])};
    out[0] = out[1] = out[2] = out[3] = 0.0;
#pragma unroll 1
    for (int S = neg;; S = (S - 1) & neg) {  // every subset S of the negative axes
        double r[4];
        cut_term(gl, R, t, (has & ~neg) | S, r);
        const double sg = (__popc(S) & 1) ? -1.0 : 1.0;
        out[0] += sg * r[0];
        for (int k = 0; k < 3; ++k) out[1 + k] += sg * (((S >> k) & 1) ? -r[1 + k] : r[1 + k]);
        if (S == 0) break;
    }
}

// One shared-region term: the walls w[0..m-1] at distances d[] cut W; the
// repulsion K_n (R_c - |cbar|) |W| along the centroid's direction, signed,
// goes to f, and its component along each wall's normal to that wall.
__device__ void overlap_term(const double *wall_n, const double *gl, double Rc, double Kn, int m, const int *w,
                             const double *d, double sign, double vol, double *f, double *react)
{
    const double th[3] = {d[0], d[1], m == 3 ? d[2] : 0.0};
    double cut[4];
    ball_cut(gl, Rc, th, m == 3 ? 7 : 3, cut);
    const double V = cut[0];
    if (!(V > 0.0)) return;
    const double cb[3] = {cut[1] / V, cut[2] / V, m == 3 ? cut[3] / V : 0.0};  // along -n of each wall
    const double rb = sqrt((cb[0] * cb[0] + cb[1] * cb[1]) + cb[2] * cb[2]);
    if (!(rb > 0.0)) return;
    const double g = sign * Kn * (Rc - rb) * V / rb;
    for (int k = 0; k < m; ++k) {
        const double *nk = wall_n + 3 * w[k];
        for (int a = 0; a < 3; ++a) {
            const double fa = g * cb[k] * nk[a];
            f[a] += fa;
            react[3 * w[k] + a] -= fa * vol;
        }
    }
}

// Inclusion-exclusion over the walls the node touches (Sec. 4.1.1): minus the
// region shared by every orthogonal pair, plus the region shared by every
// mutually orthogonal triple.  Out of line: few nodes ever touch two walls.
__device__ __forceinline__ double3 wall_overlap_terms(const double *wall_pos, const double *wall_n, const double *gl,
                                                   int nw, double Rc, double Kn, double px, double py, double pz,
                                                   double vol, double *react)
{
    int w[PD_MAX_WALLS];
    double d[PD_MAX_WALLS];
    int nt = 0;
    for (int l = 0; l < nw; ++l) {
        const double *n = wall_n + 3 * l, *q = wall_pos + 3 * l;
        const double dl = dadd(dadd(dmul(px - q[0], n[0]), dmul(py - q[1], n[1])), dmul(pz - q[2], n[2]));
        if (dl < Rc && dl > -Rc) { w[nt] = l; d[nt] = dl; ++nt; }
    }
    double f[3] = {0.0, 0.0, 0.0};
#pragma unroll 1
    for (int s = 0; s < nt; ++s)
#pragma unroll 1
        for (int t = s + 1; t < nt; ++t) {
            const double *ns = wall_n + 3 * w[s], *nu = wall_n + 3 * w[t];
            if (fabs(ns[0] * nu[0] + ns[1] * nu[1] + ns[2] * nu[2]) > 1e-9) continue;
            const int w2[2] = {w[s], w[t]};
            const double d2[2] = {d[s], d[t]};
            overlap_term(wall_n, gl, Rc, Kn, 2, w2, d2, -1.0, vol, f, react);
#pragma unroll 1
            for (int r = t + 1; r < nt; ++r) {
                const double *nr = wall_n + 3 * w[r];
                if (fabs(ns[0] * nr[0] + ns[1] * nr[1] + ns[2] * nr[2]) > 1e-9) continue;
                if (fabs(nu[0] * nr[0] + nu[1] * nr[1] + nu[2] * nr[2]) > 1e-9) continue;
                const int w3[3] = {w[s], w[t], w[r]};
                const double d3[3] = {d[s], d[t], d[r]};
                overlap_term(wall_n, gl, Rc, Kn, 3, w3, d3, 1.0, vol, f, react);
            }
        }
    return make_double3(f[0], f[1], f[2]);
}

// Wall forces on one node (Sec. 4.1): the cap repulsion and its damping; with
// WX (the kernels launched when friction or inclusion-exclusion is on) also the
// wall friction and the multi-wall terms, which other kernels do not carry.
template <bool WX>
__device__ __forceinline__ unsigned wall_force(const StepParams &p, const double *wp, double px, double py, double pz,
                                               double vol, double vx, double vy, double vz, double &fx,
                                               double &fy, double &fz, double *react)
{
    unsigned e = 0;
    int touching = 0;
    for (int l = 0; l < p.walls.nw; ++l) {
        const double nx = p.walls.n[l][0], ny = p.walls.n[l][1], nz = p.walls.n[l][2];
        const double *w = wp + 3 * l;
        double d = dadd(dadd(dmul(px - w[0], nx), dmul(py - w[1], ny)), dmul(pz - w[2], nz));
        if (!(d < p.Rc)) continue;
        if (d <= -p.Rc) { e |= PDE_WALL; continue; }
        double hc = p.Rc - d;
        double vcap = (M_PI / 3.0) * hc * hc * (2.0 * p.Rc + d);
        double q = p.Rc * p.Rc - d * d;
        double zbar = (M_PI / 4.0) * q * q / vcap;
        double mag = p.Kn * (p.Rc - zbar) * vcap;
        if (p.beta_d > 0.0)  // damping: the cap moves with the wall (Sec. 4.1 substitution)
            mag += p.beta_d * (((p.walls.v[l][0] - vx) * nx + (p.walls.v[l][1] - vy) * ny) +
                               (p.walls.v[l][2] - vz) * nz) * vcap;
        fx += mag * nx; fy += mag * ny; fz += mag * nz;
        react[3 * l + 0] -= mag * nx * vol;
        react[3 * l + 1] -= mag * ny * vol;
        react[3 * l + 2] -= mag * nz * vol;
        if (WX && p.mu > 0.0) {  // stick-slip friction against the sliding of the node along the wall
            const double rx = vx - p.walls.v[l][0], ry = vy - p.walls.v[l][1], rz = vz - p.walls.v[l][2];
            const double vn = (rx * nx + ry * ny) + rz * nz;
            const double tx = rx - vn * nx, ty = ry - vn * ny, tz = rz - vn * nz;
            const double vt = sqrt((tx * tx + ty * ty) + tz * tz);
            if (vt > 0.0) {
                const double slip = p.mu * p.Kn * (p.Rc - zbar) * vcap;
                const double stick = p.dt_f > 0.0 ? p.rho * vt / p.dt_f : INFINITY;
                const double fm = stick < slip ? stick : slip;
                fx -= fm * tx / vt; fy -= fm * ty / vt; fz -= fm * tz / vt;
                react[3 * l + 0] += fm * tx / vt * vol;
                react[3 * l + 1] += fm * ty / vt * vol;
                react[3 * l + 2] += fm * tz / vt * vol;
            }
        }
        ++touching;
    }
    if (WX && p.wall_overlap && touching >= 2) {
        const double3 o = wall_overlap_terms(wp, p.wall_n, p.gl, p.walls.nw, p.Rc, p.Kn, px, py, pz, vol,
                                             react);
        fx += o.x; fy += o.y; fz += o.z;
    }
    return e;
}

// x_lo rides in the spare lanes of the u records as BF16: R1.w = (x_lo.x, x_lo.y),
// R2.w = (x_lo.z, 0).  BF16 keeps 8 bits of x_lo, so x is known to 2^-32 |x|
// (x is stored relative to the centre of the bounding box).
__device__ __forceinline__ void xl_unpack(float w1, float w2, float *xl)
{
    const uint32_t a = __float_as_uint(w1), b = __float_as_uint(w2);
    xl[0] = __uint_as_float(a << 16);
    xl[1] = __uint_as_float(a & 0xffff0000u);
    xl[2] = __uint_as_float(b << 16);
}

// The three record slots of neighbour j (mixed path), in the layout PD_PLANES
// selects: (x_hi, c V), (u_hi, x_lo.xy packed), (u_lo, x_lo.z packed).
__device__ __forceinline__ void gather_record(const StepParams &p, int32_t j, float4 &a0, float4 &a1, float4 &a2)
{
#if PD_PLANES == 2
    a0 = __ldg(p.xh4 + j);
    // the node's u pair is 32-byte aligned (u0 even): one 256-bit read-only load
    const float4 *q = p.uh_in + 2 * (int64_t)j;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a1.x), "=f"(a1.y), "=f"(a1.z), "=f"(a1.w), "=f"(a2.x), "=f"(a2.y), "=f"(a2.z), "=f"(a2.w)
        : "l"(q));
#elif PD_PLANES == 1
    a0 = __ldg(p.xh4 + j);
    a1 = __ldg(p.uh_in + j);
    a2 = __ldg(p.ul_in + j);
#else
    const float4 *r = p.xh4 + 3 * (int64_t)j;  // one 48-byte record
    a0 = __ldg(r);
    a1 = __ldg(r + 1);
    a2 = __ldg(r + 2);
#endif
}

// One bond of the mixed path (Eq. pmb with the bond memory of Eq. peri-damage):
// records o* of the row's node and a* of the neighbour.
template <bool FLAG = false>
__device__ __forceinline__ void bond_mixed(const StepParams &p, int64_t k, const float4 &o0, const float4 &o1,
                                           const float4 &o2, const float *ol, const float4 &a0, const float4 &a1,
                                           const float4 &a2, float &fbx, float &fby, float &fbz)
{
    float al[3];
    xl_unpack(a1.w, a2.w, al);
    const float xx = (a0.x - o0.x) + (al[0] - ol[0]);
    const float xy = (a0.y - o0.y) + (al[1] - ol[1]);
    const float xz = (a0.z - o0.z) + (al[2] - ol[2]);
    const float ex = (a1.x - o1.x) + (a2.x - o2.x);
    const float ey = (a1.y - o1.y) + (a2.y - o2.y);
    const float ez = (a1.z - o1.z) + (a2.z - o2.z);
    const float yx = xx + ex, yy = xy + ey, yz = xz + ez;
    const float L2 = fmaf(xx, xx, fmaf(xy, xy, xz * xz));
    const float y2 = fmaf(yx, yx, fmaf(yy, yy, yz * yz));
    const float num = fmaf(ex, xx + yx, fmaf(ey, xy + yy, ez * (xz + yz)));
    const float rL = rsqrtf(L2), ry = rsqrtf(y2);
    const float s = __fdividef(num * rL, fmaf(y2, ry, L2 * rL));
    const bool brk = p.break_mode ? (fabsf(s) > p.s0f) : (s > p.s0f);
    if (brk) {
        atomicOr(p.brk + (k >> 5), 1u << (k & 31));
        // the tiled path also carries the flag in bit 15 of the 16-bit local index,
        // the global mixed path in bit 31 of the index
        if (FLAG) atomicOr((unsigned int *)(p.lcol) + (k >> 1), 0x8000u << (16 * (int)(k & 1)));
        if (p.colf) atomicOr((unsigned int *)p.colf + k, 0x80000000u);
    } else {
        float g = a0.w * s * ry;  // a0.w holds c V_j
        if (p.conic) g *= p.delta_f - L2 * rL;
        fbx = fmaf(g, yx, fbx);
        fby = fmaf(g, yy, fby);
        fbz = fmaf(g, yz, fbz);
    }
}

// One slot of the global mixed path.  raw = neighbour index with the broken flag
// in bit 31.  The bond is evaluated whatever the flag and its force masked, so
// that intact and broken slots take the same instruction stream; a bond that
// breaks now flags its slot in both copies of the bond memory.
__device__ __forceinline__ void bond_mixed_flagged(const StepParams &p, int k, int32_t raw, const float4 &o0,
                                                   const float4 &o1, const float4 &o2, const float *ol,
                                                   const float4 &a0, const float4 &a1, const float4 &a2, float &fbx,
                                                   float &fby, float &fbz)
{
    // The x and y components go through packed FP32x2 instructions (Blackwell):
    // a 16-byte load leaves them in a register pair, and each lane of a packed
    // add/mul/fma rounds exactly like the scalar instruction, so this is the same
    // arithmetic, operation for operation, as the scalar form of bond_mixed.
    float al[3];
    xl_unpack(a1.w, a2.w, al);
    const float2 xxy = __fadd2_rn(__fadd2_rn(make_float2(a0.x, a0.y), make_float2(-o0.x, -o0.y)),
                                  __fadd2_rn(make_float2(al[0], al[1]), make_float2(-ol[0], -ol[1])));
    const float xz = (a0.z - o0.z) + (al[2] - ol[2]);
    const float2 exy = __fadd2_rn(__fadd2_rn(make_float2(a1.x, a1.y), make_float2(-o1.x, -o1.y)),
                                  __fadd2_rn(make_float2(a2.x, a2.y), make_float2(-o2.x, -o2.y)));
    const float ez = (a1.z - o1.z) + (a2.z - o2.z);
    const float2 yxy = __fadd2_rn(xxy, exy);
    const float yz = xz + ez;
    const float L2 = fmaf(xxy.x, xxy.x, fmaf(xxy.y, xxy.y, xz * xz));
    const float y2 = fmaf(yxy.x, yxy.x, fmaf(yxy.y, yxy.y, yz * yz));
    const float2 txy = __fadd2_rn(xxy, yxy);
    const float num = fmaf(exy.x, txy.x, fmaf(exy.y, txy.y, ez * (xz + yz)));
    const float rL = rsqrtf(L2), ry = rsqrtf(y2);
    const float s = __fdividef(num * rL, fmaf(y2, ry, L2 * rL));
    const bool intact = raw >= 0;
    const bool brk = intact && (p.break_mode ? (fabsf(s) > p.s0f) : (s > p.s0f));
    if (brk) {
        p.colf[k] = (int32_t)((uint32_t)raw | 0x80000000u);
        atomicOr(p.brk + (k >> 5), 1u << (k & 31));
    }
    // a0.w holds c V_j (the record's volume slot is scaled at bond build); the
    // conic micromodulus multiplies by delta - |xi| (uniform branch).  The mask
    // comes last, so that a masked slot adds exactly zero whatever its arithmetic
    // gave (a padding slot may even gather the row's own record)
    float g = a0.w * s * ry;
    if (p.conic) g *= p.delta_f - L2 * rL;
    g = (intact && !brk) ? g : 0.f;
    const float2 f = __ffma2_rn(make_float2(g, g), yxy, make_float2(fbx, fby));
    fbx = f.x;
    fby = f.y;
    fbz = fmaf(g, yz, fbz);
}

// ---- Each bond once (mixed path, two passes) ---------------------------------
// Eq. pmb is pairwise antisymmetric: with y the current bond vector from i to j,
// the force density on i is c s V_j y/|y| and the one on j is -c s V_i y/|y|.  Pass
// 1 evaluates every bond from its lower-index end i (the slots of row i whose
// neighbour index is larger): it adds its own term and leaves the factor
// c V_i s/|y| for j at the mirror slot (the same bond seen from j).  Pass 2 walks
// each row's other slots, forms y from j's side (formed from the two records by
// the same operations with the roles swapped, so it is exactly -y) and applies
// the stored factor.  Every sum runs in a fixed order: results are reproducible.

// y = x_j + u_j - x_i - u_i from the records of the row's node (o*) and the
// neighbour (a*), operation by operation as in bond_mixed_flagged
__device__ __forceinline__ void pair_y(const float4 &o0, const float4 &o1, const float4 &o2, const float *ol,
                                       const float4 &a0, const float4 &a1, const float4 &a2, float2 &yxy, float &yz,
                                       float2 &xxy, float &xz, float2 &exy, float &ez)
{
    float al[3];
    xl_unpack(a1.w, a2.w, al);
    xxy = __fadd2_rn(__fadd2_rn(make_float2(a0.x, a0.y), make_float2(-o0.x, -o0.y)),
                     __fadd2_rn(make_float2(al[0], al[1]), make_float2(-ol[0], -ol[1])));
    xz = (a0.z - o0.z) + (al[2] - ol[2]);
    exy = __fadd2_rn(__fadd2_rn(make_float2(a1.x, a1.y), make_float2(-o1.x, -o1.y)),
                     __fadd2_rn(make_float2(a2.x, a2.y), make_float2(-o2.x, -o2.y)));
    ez = (a1.z - o1.z) + (a2.z - o2.z);
    yxy = __fadd2_rn(xxy, exy);
    yz = xz + ez;
}

// Pass 1, slot k of row i (neighbour j > i), mirror slot m: stretch, breaking of
// both slots, the row's own term, and the partner's factor at tb[m].
__device__ __forceinline__ void bond_pair_upper(const StepParams &p, int k, int m, int32_t raw, const float4 &o0,
                                                const float4 &o1, const float4 &o2, const float *ol, const float4 &a0,
                                                const float4 &a1, const float4 &a2, float &fbx, float &fby, float &fbz)
{
    float2 yxy, xxy, exy;
    float yz, xz, ez;
    pair_y(o0, o1, o2, ol, a0, a1, a2, yxy, yz, xxy, xz, exy, ez);
    const float L2 = fmaf(xxy.x, xxy.x, fmaf(xxy.y, xxy.y, xz * xz));
    const float y2 = fmaf(yxy.x, yxy.x, fmaf(yxy.y, yxy.y, yz * yz));
    const float2 txy = __fadd2_rn(xxy, yxy);
    const float num = fmaf(exy.x, txy.x, fmaf(exy.y, txy.y, ez * (xz + yz)));
    const float rL = rsqrtf(L2), ry = rsqrtf(y2);
    const float s = __fdividef(num * rL, fmaf(y2, ry, L2 * rL));
    const bool intact = raw >= 0;
    const bool brk = intact && (p.break_mode ? (fabsf(s) > p.s0f) : (s > p.s0f));
    if (brk) {  // the bond memory of both directed slots, in both copies
        p.colf[k] = (int32_t)((uint32_t)raw | 0x80000000u);
        atomicOr((unsigned int *)p.colf + m, 0x80000000u);
        atomicOr(p.brk + (k >> 5), 1u << (k & 31));
        atomicOr(p.brk + (m >> 5), 1u << (m & 31));
    }
    float t = (intact && !brk) ? s * ry : 0.f;
    if (p.conic) t *= p.delta_f - L2 * rL;
    const float gi = a0.w * t;  // a0.w = c V_j
    const float2 f = __ffma2_rn(make_float2(gi, gi), yxy, make_float2(fbx, fby));
    fbx = f.x;
    fby = f.y;
    fbz = fmaf(gi, yz, fbz);
    p.tb[m] = o0.w * t;  // o0.w = c V_i: the factor of j's term
}

// Pass 1: upper slots of every row; the row's partial force goes to fup.
template <int G>
__global__ void __launch_bounds__(STEP_THREADS, PD_MINB_GLOBAL) k_pairs_upper(const StepParams p)
{
    constexpr int GPB = STEP_THREADS / G;
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    if (segment_doomed(p)) return;
    for (int64_t r0 = (int64_t)blockIdx.x * GPB; r0 < p.n; r0 += (int64_t)gridDim.x * GPB) {
        const int64_t row = r0 + grp;
        float fbx = 0.f, fby = 0.f, fbz = 0.f;
        if (row < p.n) {
            const float4 o0 = __ldg(p.xh4 + RECX * row), o1 = __ldg(p.uh_in + REC * row),
                         o2 = __ldg(p.ul_in + REC * row);
            float ol[3];
            xl_unpack(o1.w, o2.w, ol);
            const int i0 = __ldg(p.split + row), i1 = (int)__ldg(p.rowptr + row + 1);
            for (int k = i0 + gl; k < i1; k += PD_INFLIGHT * G) {
                int32_t raw[PD_INFLIGHT], mk[PD_INFLIGHT];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q) {
                    // a slot past the row end reuses the first slot's node and writes nothing
                    const int kq = k + q * G;
                    const bool ok = q == 0 || kq < i1;
                    raw[q] = ok ? ld_slot(p.colf + kq) : raw[0];
                    mk[q] = ok ? __ldg(p.mir + kq) : -1;
                }
                float4 a0[PD_INFLIGHT], a1[PD_INFLIGHT], a2[PD_INFLIGHT];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q) {
                    gather_record(p, raw[q] & 0x7fffffff, a0[q], a1[q], a2[q]);
                }
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q)
                    if (mk[q] >= 0)
                        bond_pair_upper(p, k + q * G, mk[q], raw[q], o0, o1, o2, ol, a0[q], a1[q], a2[q], fbx, fby,
                                        fbz);
            }
        }
        fbx = group_sum<G>(fbx);
        fby = group_sum<G>(fby);
        fbz = group_sum<G>(fbz);
        if (row < p.n && gl == 0) p.fup[row] = make_float4(fbx, fby, fbz, 0.f);
    }
}

// u of node i in FP64: the double-float state of the mixed path, or the FP64 array
template <bool MIXED>
__device__ __forceinline__ dbl4 load_u_t(const StepParams &p, int64_t i)
{
    dbl4 r;
    if (MIXED) {
        const float4 h = p.uh_in[REC * i], l = p.ul_in[REC * i];
        r.x = df_to_double(df{h.x, l.x});
        r.y = df_to_double(df{h.y, l.y});
        r.z = df_to_double(df{h.z, l.z});
        r.w = 0.0;
    } else {
        r = p.u_in[i];
    }
    return r;
}

// Component c = gl of the mixed-path Verlet update of one row.
__device__ __forceinline__ unsigned epilogue_component(const StepParams &p, int64_t row, int c, float Fx, float Fy,
                                                       float Fz, const float4 &uh, const float4 &ul,
                                                       const float4 &vh, const float4 &vl, float &vc2)
{
    unsigned err = 0;
    const float F = c == 0 ? Fx : (c == 1 ? Fy : Fz);
    if (!isfinite(F)) err |= PDE_NONFINITE;
    const float a = (F + p.bf[c]) * p.inv_rho_f;
    float *afc = (float *)(p.af + row) + c;
    if (p.mode == MODE_FORCES) {
        *afc = a;
        if (p.F_out) ((double *)(p.F_out + row))[c] = (double)F;
        return err;
    }
    const df hdt{p.hdt_hi, p.hdt_lo};
    const float vhc = c == 0 ? vh.x : (c == 1 ? vh.y : vh.z);
    const float vlc = c == 0 ? vl.x : (c == 1 ? vl.y : vl.z);
    // every pair the step stores, or would store when split into single-step
    // calls, is put on the FP64 grid
    df v = df_on_fp64_grid(df_add(df{vhc, vlc}, df_mul_f(hdt, a)));
    if (p.mode == MODE_FULL) {
        v = df_on_fp64_grid(df_add(v, df_mul_f(hdt, a)));
        const float uhc = c == 0 ? uh.x : (c == 1 ? uh.y : uh.z);
        const float ulc = c == 0 ? ul.x : (c == 1 ? ul.y : ul.z);
        const df u = df_on_fp64_grid(df_add(df{uhc, ulc}, df_mul(df{p.dt_hi, p.dt_lo}, v)));
        ((float *)(p.uh_out + REC * row))[c] = u.hi;
        ((float *)(p.ul_out + REC * row))[c] = u.lo;
        if (c == 0) {  // packed x_lo travels with the record
            ((float *)(p.uh_out + REC * row))[3] = uh.w;
            ((float *)(p.ul_out + REC * row))[3] = ul.w;
        }
        vc2 = v.hi * v.hi;
        if (!isfinite(v.hi) || !isfinite(u.hi)) err |= PDE_NONFINITE;
    } else {
        *afc = a;
    }
    ((float *)(p.vh + row))[c] = v.hi;
    ((float *)(p.vl + row))[c] = v.lo;
    return err;
}

// Mixed-path epilogue spread over the group: lane c (0, 1, 2) updates component
// c of the node's acceleration, velocity and displacement.  Every lane of the
// warp calls it (inactive rows included) so that the shuffles that broadcast a
// wall force and sum |v|^2 are uniform.
template <int G, bool WX>
__device__ __forceinline__ unsigned epilogue_lanes(const StepParams &p, const double *wp, int64_t row, bool active,
                                                   int gl, float Fx,
                                                   float Fy, float Fz, const float4 &oxh, const float4 &uh,
                                                   const float4 &ul, const float4 &vh, const float4 &vl,
                                                   double *react, float &vmax2)
{
    unsigned err = 0;
    if (p.walls.nw) {  // uniform: a kernel parameter
        float wx = 0.f, wy = 0.f, wz = 0.f;
        if (active && gl == 0) {
            const float px = oxh.x + uh.x, py = oxh.y + uh.y, pz = oxh.z + uh.z;
            const float cx = (float)p.centre[0], cy = (float)p.centre[1], cz = (float)p.centre[2];
            bool near = false;
            for (int l = 0; l < p.walls.nw; ++l) {
                const double *w = wp + 3 * l;
                const float qx = (float)w[0] - cx, qy = (float)w[1] - cy, qz = (float)w[2] - cz;
                const float d = (px - qx) * (float)p.walls.n[l][0] + (py - qy) * (float)p.walls.n[l][1] +
                                (pz - qz) * (float)p.walls.n[l][2];
                const float margin = 1e-6f * (fabsf(px) + fabsf(py) + fabsf(pz) + fabsf(qx) + fabsf(qy) +
                                              fabsf(qz) + fabsf(cx) + fabsf(cy) + fabsf(cz));
                near |= d < p.Rc_f + margin;
            }
            if (near) {
                const dbl4 ox = p.x4[row];
                const double ux = df_to_double(df{uh.x, ul.x}), uy = df_to_double(df{uh.y, ul.y}),
                             uz = df_to_double(df{uh.z, ul.z});
                double fx = 0.0, fy = 0.0, fz = 0.0;
                err |= wall_force<WX>(p, wp, dadd(ox.x, ux), dadd(ox.y, uy), dadd(ox.z, uz), ox.w, df_to_double(df{vh.x, vl.x}),
                                  df_to_double(df{vh.y, vl.y}), df_to_double(df{vh.z, vl.z}), fx, fy, fz, react);
                wx = (float)fx; wy = (float)fy; wz = (float)fz;
            }
        }
        const int leader = (int)(threadIdx.x & 31) & ~(G - 1);
        Fx += __shfl_sync(0xffffffffu, wx, leader);
        Fy += __shfl_sync(0xffffffffu, wy, leader);
        Fz += __shfl_sync(0xffffffffu, wz, leader);
    }
    float vc2 = 0.f;  // v_c^2 of this lane's component (0 on lanes 3.. and inactive rows)
    if (active && gl < 3) err |= epilogue_component(p, row, gl, Fx, Fy, Fz, uh, ul, vh, vl, vc2);
    // |v|^2 of the row: lanes 0..3 of the group form an aligned quad (G >= 4)
    float v2 = vc2 + __shfl_xor_sync(0xffffffffu, vc2, 1);
    v2 += __shfl_xor_sync(0xffffffffu, v2, 2);
    vmax2 = fmaxf(vmax2, v2);
    return err;
}

// One contact candidate q of row i (Sec. 3.2, the self-contact law, and the
// normal damping of Sec. 3.3): false when the pair does not touch or is still
// bonded; otherwise (gx, gy, gz) = its force density on i.  The predicate is
// evaluated in FP64 without FMA, so contact pair sets are exact.
template <bool MIXED>
__device__ __forceinline__ bool contact_term(const StepParams &p, int64_t q, const dbl4 &ox, double pix, double piy,
                                             double piz, int gi, double R2, double &gx, double &gy, double &gz)
{
    const int2 cj = p.cand[q];
    const int j = cj.x;
    if (cj.y >= 0) {
        const uint32_t w = *((volatile uint32_t *)(p.brk + (cj.y >> 5)));
        if (!((w >> (cj.y & 31)) & 1u)) return false;  // bond intact
    }
    const dbl4 xj = p.x4[j], uj = load_u_t<MIXED>(p, j);
    const double dx = dadd(xj.x, uj.x) - pix;
    const double dy = dadd(xj.y, uj.y) - piy;
    const double dz = dadd(xj.z, uj.z) - piz;
    const double d2 = dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz));
    if (!(d2 < R2)) return false;
    const double dn = sqrt(d2);
    if (dn == 0.0) return false;
    double mag;
    const double xx = xj.x - ox.x, xy = xj.y - ox.y, xz = xj.z - ox.z;
    const double L = sqrt(dadd(dadd(dmul(xx, xx), dmul(xy, xy)), dmul(xz, xz)));
    if (p.grain[j] != gi || L >= p.Rc) {
        mag = -p.Kn * (p.Rc - dn);
    } else {
        const double sr = (dn - L) / L;
        mag = (p.conic ? p.c * (p.delta - L) : p.c) * (sr < 0.0 ? sr : 0.0);
    }
    const double gm = mag * xj.w / dn;
    gx = gm * dx; gy = gm * dy; gz = gm * dz;
    if (p.pair_diss) {  // damping and friction of this pair, computed before the step by k_pair_damping
        if (MIXED) {
            const float4 f = ((const float4 *)p.cand_fd)[q];
            gx += f.x; gy += f.y; gz += f.z;
        } else {
            const dbl4 f = ((const dbl4 *)p.cand_fd)[q];
            gx += f.x; gy += f.y; gz += f.z;
        }
    }
    return true;
}

// Contact force density on `row` (Sec. 3.2 and the self-contact law, with the
// pair damping and friction of Sec. 3.3).  The group's lanes evaluate the
// candidates G at a time, and every lane adds the terms in list order through an
// ordered shuffle chain.  The lists are sorted by partner index and a candidate
// that does not touch adds exactly zero, so the result is the sum over the
// touching pairs alone in ascending partner order: an evaluation at a given state
// gives the same bits whichever rebuild (and skin superset) made the list.  All
// lanes of the warp call it (inactive rows with active = false).
template <int G, bool MIXED>
__device__ __forceinline__ void contact_sum(const StepParams &p, int64_t row, bool active, int gl, double &cx,
                                            double &cy, double &cz)
{
    cx = cy = cz = 0.0;
    int64_t c0 = 0, c1 = 0;
    if (active && p.contact) {
        c0 = p.cand_ptr[row];
        c1 = p.cand_ptr[row + 1];
    }
    const int nch = (int)((c1 - c0 + G - 1) / G);
    const int nmax = __reduce_max_sync(0xffffffffu, nch);  // warp-uniform trip count
    if (nmax == 0) return;
    dbl4 ox = dbl4{0.0, 0.0, 0.0, 0.0};
    double pix = 0.0, piy = 0.0, piz = 0.0;
    int gi = 0;
    if (nch > 0) {
        ox = p.x4[row];
        const dbl4 ou = load_u_t<MIXED>(p, row);
        pix = dadd(ox.x, ou.x); piy = dadd(ox.y, ou.y); piz = dadd(ox.z, ou.z);
        gi = p.grain[row];
    }
    const double R2 = dmul(p.Rc, p.Rc);
    for (int t = 0; t < nmax; ++t) {
        const int64_t q = c0 + (int64_t)t * G + gl;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        if (q < c1 && !contact_term<MIXED>(p, q, ox, pix, piy, piz, gi, R2, gx, gy, gz)) gx = gy = gz = 0.0;
#pragma unroll
        for (int l = 0; l < G; ++l) {
            cx += __shfl_sync(0xffffffffu, gx, l, G);
            cy += __shfl_sync(0xffffffffu, gy, l, G);
            cz += __shfl_sync(0xffffffffu, gz, l, G);
        }
    }
}

// velocity of node i in FP64 (double-float pair on the mixed path)
template <bool MIXED>
__device__ __forceinline__ void load_v_t(const StepParams &p, int64_t i, double &vx, double &vy, double &vz)
{
    if (MIXED) {
        const float4 h = p.vh[i], l = p.vl[i];
        vx = df_to_double(df{h.x, l.x}); vy = df_to_double(df{h.y, l.y}); vz = df_to_double(df{h.z, l.z});
    } else {
        const dbl4 v = p.v[i];
        vx = v.x; vy = v.y; vz = v.z;
    }
}

// The velocity-dependent pair forces of every contact candidate, summed:
// - normal damping (Sec. 3.3), read as the dissipative linear law
//   beta_d ((v_j - v_i) . e) e V_j;
// - stick-slip friction (Sec. 3.3, Eq. regularized-friction), read as
//   -min(rho |v_t| / (dt (V_i + V_j)), mu f_r) V_j v_t / |v_t| with v_t the part
//   of v_i - v_j across e and f_r the pair's repulsion per volume squared: the
//   slip branch opposes the slip, and the stick branch, divided by V_i + V_j,
//   is antisymmetric and stops an isolated pair's sliding in one step.
// Runs before the step kernel, while no kernel writes velocities, so that the
// step kernel (which updates v in place) reads a consistent half-step velocity
// field; candidates that do not touch get zero, and the step kernel adds the
// term only to pairs it accepts.
template <bool MIXED>
__device__ __forceinline__ void pair_damping_rows(const StepParams &p, int64_t first, int64_t stride)
{
    const double R2 = dmul(p.Rc, p.Rc);
    for (int64_t i = first; i < p.n; i += stride) {
        const int64_t c0 = p.cand_ptr[i], c1 = p.cand_ptr[i + 1];
        if (c1 <= c0) continue;
        const dbl4 ox = p.x4[i], ou = load_u_t<MIXED>(p, i);
        const double pix = dadd(ox.x, ou.x), piy = dadd(ox.y, ou.y), piz = dadd(ox.z, ou.z);
        const int gi = p.grain[i];
        double vix, viy, viz;
        load_v_t<MIXED>(p, i, vix, viy, viz);
        for (int64_t q = c0; q < c1; ++q) {
            const int j = p.cand[q].x;
            const dbl4 xj = p.x4[j], uj = load_u_t<MIXED>(p, j);
            const double dx = dadd(xj.x, uj.x) - pix;
            const double dy = dadd(xj.y, uj.y) - piy;
            const double dz = dadd(xj.z, uj.z) - piz;
            const double d2 = dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz));
            double fx = 0.0, fy = 0.0, fz = 0.0;
            if (d2 < R2 && d2 > 0.0) {
                const double dn = sqrt(d2);
                const double ex = dx / dn, ey = dy / dn, ez = dz / dn;
                double vjx, vjy, vjz;
                load_v_t<MIXED>(p, j, vjx, vjy, vjz);
                if (p.beta_d > 0.0) {
                    const double w = (vjx - vix) * ex + (vjy - viy) * ey + (vjz - viz) * ez;
                    const double g = p.beta_d * w * xj.w;
                    fx = g * ex; fy = g * ey; fz = g * ez;
                }
                if (p.mu > 0.0) {
                    // the repulsion of the contact law (spring, or the PD-repulsive
                    // law of a once-bonded same-grain pair)
                    const double xx = xj.x - ox.x, xy = xj.y - ox.y, xz = xj.z - ox.z;
                    const double L = sqrt(dadd(dadd(dmul(xx, xx), dmul(xy, xy)), dmul(xz, xz)));
                    double fr;
                    if (p.grain[j] != gi || L >= p.Rc) {
                        fr = p.Kn * (p.Rc - dn);
                    } else {
                        const double sr = (dn - L) / L;
                        fr = sr < 0.0 ? -(p.conic ? p.c * (p.delta - L) : p.c) * sr : 0.0;
                    }
                    const double rx = vix - vjx, ry = viy - vjy, rz = viz - vjz;
                    const double vn = (rx * ex + ry * ey) + rz * ez;
                    const double tx = rx - vn * ex, ty = ry - vn * ey, tz = rz - vn * ez;
                    const double vt = sqrt((tx * tx + ty * ty) + tz * tz);
                    if (vt > 0.0) {
                        const double slip = p.mu * fr;
                        const double stick = p.dt_f > 0.0 ? p.rho * vt / (p.dt_f * (ox.w + xj.w)) : INFINITY;
                        const double fm = stick < slip ? stick : slip;
                        fx -= fm * (tx / vt) * xj.w;
                        fy -= fm * (ty / vt) * xj.w;
                        fz -= fm * (tz / vt) * xj.w;
                    }
                }
            }
            if (MIXED)
                ((float4 *)p.cand_fd)[q] = make_float4((float)fx, (float)fy, (float)fz, 0.f);
            else
                ((dbl4 *)p.cand_fd)[q] = dbl4{fx, fy, fz, 0.0};
        }
    }
}

template <bool MIXED>
__global__ void k_pair_damping(const StepParams p)
{
    pair_damping_rows<MIXED>(p, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Tile staging of the mixed path: the records of the nodes a tile touches.
struct TileView {
    const float4 *s0, *s1, *s2;  // shared copies of xh4, uh_in, ul_in for the tile's list
    bool on;                     // false: gather from global memory
};

// Steps 1-4 for one row owned by a group of G lanes (all lanes call; inactive
// groups pass active = false and still join the shuffles).
template <int G, bool MIXED, bool WX = false, bool PAIRS = false>
__device__ __forceinline__ void process_row(const StepParams &p, const double *wp, int64_t row, bool active, int gl,
                                            int lrow,
                                            const TileView &tv, double *react, unsigned &err, float &vmax2f,
                                            double &vmax2)
{
#define load_u(P, I) load_u_t<MIXED>(P, I)
    // ---- 1. bonds
    float fbx = 0.f, fby = 0.f, fbz = 0.f;
    double fdx = 0.0, fdy = 0.0, fdz = 0.0;
    if (active) {
        const int64_t k0 = p.rowptr[row], k1 = p.rowptr[row + 1];
        if (PAIRS) {
            // pass 2: the slots whose bond pass 1 evaluated from the other end
            // (neighbour index below the row's); their factors are in tb
            const float4 o0 = __ldg(p.xh4 + RECX * row), o1 = __ldg(p.uh_in + REC * row),
                         o2 = __ldg(p.ul_in + REC * row);
            float ol[3];
            xl_unpack(o1.w, o2.w, ol);
            const int i0 = (int)k0, i1 = __ldg(p.split + row);
            for (int k = i0 + gl; k < i1; k += PD_INFLIGHT * G) {
                int32_t raw[PD_INFLIGHT];
                float g[PD_INFLIGHT];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q) {
                    const int kq = k + q * G;
                    const bool ok = q == 0 || kq < i1;
                    raw[q] = ok ? ld_slot(p.colf + kq) : raw[0];
                    g[q] = ok ? __ldcs(p.tb + kq) : 0.f;
                }
                float4 a0[PD_INFLIGHT], a1[PD_INFLIGHT], a2[PD_INFLIGHT];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q) {
                    gather_record(p, raw[q] & 0x7fffffff, a0[q], a1[q], a2[q]);
                }
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q) {
                    float2 yxy, xxy, exy;
                    float yz, xz, ez;
                    pair_y(o0, o1, o2, ol, a0[q], a1[q], a2[q], yxy, yz, xxy, xz, exy, ez);
                    const float2 f = __ffma2_rn(make_float2(g[q], g[q]), yxy, make_float2(fbx, fby));
                    fbx = f.x;
                    fby = f.y;
                    fbz = fmaf(g[q], yz, fbz);
                }
            }
        } else if (MIXED) {
            const float4 o0 = __ldg(p.xh4 + RECX * row), o1 = __ldg(p.uh_in + REC * row), o2 = __ldg(p.ul_in + REC * row);
            float ol[3];
            xl_unpack(o1.w, o2.w, ol);
            const int i0 = (int)k0, i1 = (int)k1;
#if PD_PREFETCH
            // software pipeline: the slot words of the next batch are loaded while
            // the current batch's records are gathered and evaluated, so that the
            // streamed index load and the dependent gather do not follow one
            // another on every batch
            int32_t raw[PD_INFLIGHT_PF];
            {
                const int k = i0 + gl;
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT_PF; ++q) {
                    // a slot past the row end gathers the first slot's node, flagged
                    const int kq = k + q * G;
                    raw[q] = kq < i1 ? ld_slot(p.colf + kq)
                                     : (q == 0 ? (int32_t)0x80000000u : (int32_t)((uint32_t)raw[0] | 0x80000000u));
                }
            }
            for (int k = i0 + gl; k < i1; k += PD_INFLIGHT_PF * G) {
                float4 a0[PD_INFLIGHT_PF], a1[PD_INFLIGHT_PF], a2[PD_INFLIGHT_PF];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT_PF; ++q) {
                    gather_record(p, raw[q] & 0x7fffffff, a0[q], a1[q], a2[q]);
                }
                int32_t nxt[PD_INFLIGHT_PF];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT_PF; ++q) {
                    // a slot past the row end gathers this batch's first node (a
                    // neighbour of the row), flagged: no force
                    const int kq = k + (PD_INFLIGHT_PF + q) * G;
                    nxt[q] = kq < i1 ? ld_slot(p.colf + kq) : (int32_t)((uint32_t)raw[0] | 0x80000000u);
                }
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT_PF; ++q)
                    bond_mixed_flagged(p, k + q * G, raw[q], o0, o1, o2, ol, a0[q], a1[q], a2[q], fbx, fby, fbz);
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT_PF; ++q) raw[q] = nxt[q];
            }
#else
            for (int k = i0 + gl; k < i1; k += PD_INFLIGHT * G) {
                int32_t raw[PD_INFLIGHT];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q) {
                    // a slot past the row end reuses the first slot's node, flagged
                    const int kq = k + q * G;
                    raw[q] = q == 0 ? ld_slot(p.colf + kq)
                                    : (kq < i1 ? ld_slot(p.colf + kq) : (int32_t)((uint32_t)raw[0] | 0x80000000u));
                }
                float4 a0[PD_INFLIGHT], a1[PD_INFLIGHT], a2[PD_INFLIGHT];
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q) {
                    gather_record(p, raw[q] & 0x7fffffff, a0[q], a1[q], a2[q]);
                }
#pragma unroll
                for (int q = 0; q < PD_INFLIGHT; ++q)
                    bond_mixed_flagged(p, k + q * G, raw[q], o0, o1, o2, ol, a0[q], a1[q], a2[q], fbx, fby, fbz);
            }
#endif
        } else {
            const dbl4 ox = p.x4[row], ou = p.u_in[row];
            for (int64_t k = k0 + gl; k < k1; k += G) {
                const uint32_t w = p.brk[k >> 5];
                if ((w >> (k & 31)) & 1u) continue;
                const int j = __ldg(p.col + k);
                const dbl4 a = p.x4[j], c = p.u_in[j];
                const double xx = a.x - ox.x, xy = a.y - ox.y, xz = a.z - ox.z;
                const double ex = c.x - ou.x, ey = c.y - ou.y, ez = c.z - ou.z;
                const double yx = xx + ex, yy = xy + ey, yz = xz + ez;
                const double L = sqrt(xx * xx + xy * xy + xz * xz);
                const double l = sqrt(yx * yx + yy * yy + yz * yz);
                const double s = (l - L) / L;
                const bool brk = p.break_mode ? (fabs(s) > p.s0) : (s > p.s0);
                if (brk) {
                    atomicOr(p.brk + (k >> 5), 1u << (k & 31));
                } else {
                    const double g = (p.conic ? p.c * (p.delta - L) : p.c) * s * a.w / l;
                    fdx += g * yx; fdy += g * yy; fdz += g * yz;
                }
            }
        }
    }
    __syncwarp();
    // ---- 2. contact candidates (FP64, exact predicate, ordered sum)
    double cx, cy, cz;
    contact_sum<G, MIXED>(p, row, active, gl, cx, cy, cz);
    // ---- 3. combine the group, then add pass 1's part (each bond once) and the contact sum
    if (MIXED) {
        fbx = group_sum<G>(fbx);
        fby = group_sum<G>(fby);
        fbz = group_sum<G>(fbz);
        if (PAIRS && active) {
            const float4 up = p.fup[row];
            fbx += up.x;
            fby += up.y;
            fbz += up.z;
        }
        fbx += (float)cx;
        fby += (float)cy;
        fbz += (float)cz;
    } else {
        fdx = group_sum<G>(fdx) + cx;
        fdy = group_sum<G>(fdy) + cy;
        fdz = group_sum<G>(fdz) + cz;
    }
    // ---- 4. walls and Verlet update (group leader)
    if (MIXED) {
        float4 oxh = make_float4(0.f, 0.f, 0.f, 0.f), ouh = oxh, oul = oxh, ovh = oxh, ovl = oxh;
        if (active && gl < 3) {
            oxh = __ldg(p.xh4 + RECX * row); ouh = __ldg(p.uh_in + REC * row); oul = __ldg(p.ul_in + REC * row);
            ovh = p.vh[row]; ovl = p.vl[row];
        }
        err |= epilogue_lanes<G, WX>(p, wp, row, active, gl, fbx, fby, fbz, oxh, ouh, oul, ovh, ovl, react, vmax2f);
    }
    if (!MIXED && active && gl == 0) {
        const double hdt = 0.5 * p.dt;
        double Fx = fdx, Fy = fdy, Fz = fdz;
        const dbl4 ox = p.x4[row], ou = p.u_in[row];
        const dbl4 ov = p.v[row];
        if (p.walls.nw)
            err |= wall_force<WX>(p, wp, dadd(ox.x, ou.x), dadd(ox.y, ou.y), dadd(ox.z, ou.z), ox.w, ov.x, ov.y, ov.z, Fx, Fy,
                              Fz, react);
        if (!isfinite(Fx) || !isfinite(Fy) || !isfinite(Fz)) err |= PDE_NONFINITE;
        dbl4 a;
        a.x = __ddiv_rn(dadd(Fx, p.b[0]), p.rho);
        a.y = __ddiv_rn(dadd(Fy, p.b[1]), p.rho);
        a.z = __ddiv_rn(dadd(Fz, p.b[2]), p.rho);
        a.w = 0.0;
        if (p.mode != MODE_FULL) p.acc[row] = a;
        if (p.mode == MODE_FORCES) {
            if (p.F_out) {
                dbl4 f; f.x = Fx; f.y = Fy; f.z = Fz; f.w = 0.0;
                p.F_out[row] = f;
            }
        } else {
            dbl4 v = p.v[row];
            v.x = dadd(v.x, dmul(hdt, a.x));
            v.y = dadd(v.y, dmul(hdt, a.y));
            v.z = dadd(v.z, dmul(hdt, a.z));
            if (p.mode == MODE_FULL) {
                v.x = dadd(v.x, dmul(hdt, a.x));
                v.y = dadd(v.y, dmul(hdt, a.y));
                v.z = dadd(v.z, dmul(hdt, a.z));
                dbl4 un;
                un.x = dadd(ou.x, dmul(p.dt, v.x));
                un.y = dadd(ou.y, dmul(p.dt, v.y));
                un.z = dadd(ou.z, dmul(p.dt, v.z));
                un.w = 0.0;
                p.u_out[row] = un;
                const double vv = v.x * v.x + v.y * v.y + v.z * v.z;
                vmax2 = fmax(vmax2, vv);
                if (!isfinite(vv) || !isfinite(un.x + un.y + un.z)) err |= PDE_NONFINITE;
            }
            p.v[row] = v;
        }
    }
#undef load_u
}

// Per-block partials and the finish of the step by the last block.  The max |v|
// bound goes through one atomicMax per block (a max does not depend on order);
// wall reactions are summed per block in group order, then by the last block
// with one warp per component, lanes striding over the blocks and a fixed xor
// butterfly, so the result is bitwise reproducible.  The last block also
// advances the walls and the skin bookkeeping.
template <int GPB>
__device__ __forceinline__ void block_finish(const StepParams &p, double (*s_react)[PD_MAX_WALLS * 3],
                                             double *s_vmax, unsigned &s_err, bool &s_last, unsigned err)
{
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    const int ncomp = 3 * p.walls.nw;
    double *part = p.partials + (int64_t)blockIdx.x * PART_STRIDE;
    if ((int)threadIdx.x < ncomp) {
        double s = 0.0;
        for (int g = 0; g < GPB; ++g) s += s_react[g][threadIdx.x];
        part[threadIdx.x] = s;
    } else if (threadIdx.x == 32) {
        double m = 0.0;
        for (int g = 0; g < GPB; ++g) m = fmax(m, s_vmax[g]);
        if (m > 0.0) atomicMax(p.vmax_bits, __float_as_uint(__double2float_ru(m)));
        if (s_err) atomicOr(p.err, s_err);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(p.counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < ncomp; c += STEP_THREADS / 32) {
        double s = 0.0;
        // unrolled so that the loads of several blocks' partials are in flight
        // together; the additions keep their order
#pragma unroll 8
        for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(p.partials + (int64_t)b * PART_STRIDE + c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            p.react[c] = s;
            if (p.mode != MODE_FORCES) p.impulse[c] = dadd(p.impulse[c], dmul(p.dt, s));
        }
    }
    if (threadIdx.x == 0) {
        const double vm = (double)__uint_as_float(atomicExch(p.vmax_bits, 0u));  // max |v|^2, reset
        if (p.mode == MODE_FULL) {
            const double dsp = *p.disp + p.dt * sqrt(vm);
            *p.disp = dsp;
            if (2.0 * dsp >= p.skin) *p.stale = 1;
            for (int l = 0; l < p.walls.nw; ++l)
                for (int q = 0; q < 3; ++q)
                    p.wall_pos[3 * l + q] = dadd(p.wall_pos[3 * l + q], dmul(p.dt, p.walls.v[l][q]));
        }
        *p.counter = 0u;
    }
}

// Rows in a grid-stride loop, neighbour records gathered from global memory
// (FP64 path, and the mixed path without tiles).
template <int G, bool MIXED, bool WX, bool PAIRS = false>
__global__ void __launch_bounds__(STEP_THREADS, MIXED ? PD_MINB_GLOBAL : 2) k_step(const StepParams p)
{
    constexpr int GPB = STEP_THREADS / G;
    __shared__ double s_react[GPB][PD_MAX_WALLS * 3];
    __shared__ double s_vmax[GPB];
    __shared__ unsigned s_err;
    __shared__ bool s_last;
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    if (gl == 0) {
        for (int q = 0; q < PD_MAX_WALLS * 3; ++q) s_react[grp][q] = 0.0;
    }
    if (threadIdx.x == 0) {
        s_err = 0;
        if (blockIdx.x == 0 && p.contact && *p.stale) atomicOr(p.err, (unsigned)PDE_SKIN);
    }
    if (segment_doomed(p)) return;  // uniform over the grid (see segment_doomed)
    __syncthreads();
    unsigned err = 0;
    double vmax2 = 0.0;
    float vmax2f = 0.f;
    const TileView tv{nullptr, nullptr, nullptr, false};
    for (int64_t r0 = (int64_t)blockIdx.x * GPB; r0 < p.n; r0 += (int64_t)gridDim.x * GPB) {
        const int64_t row = r0 + grp;
        process_row<G, MIXED, WX, PAIRS>(p, p.wall_pos, row, row < p.n, gl, 0, tv, s_react[grp], err, vmax2f, vmax2);
    }
    if (gl == 0) s_vmax[grp] = MIXED ? (double)vmax2f : vmax2;
    block_finish<GPB>(p, s_react, s_vmax, s_err, s_last, err);
}

// ---- Several steps in one launch ------------------------------------------------
// A run of MODE_FULL steps between two contact-list rebuilds in one cooperative
// launch: each step does what one k_step launch does (the same rows, the same
// arithmetic, the same fixed-order reductions), separated by a grid-wide barrier,
// so the trajectory is bit for bit that of one launch per step while the launch
// cost and the gap between launches are paid once per run.  Every block keeps
// its own copy of the wall positions and of the skin bookkeeping and advances
// them identically; block 0 alone writes the wall reactions and impulses, and
// at the end the walls, displacement bound and stale flag.  Even steps use the
// parameters pa (state buffers in -> out), odd steps pb (out -> in).

constexpr unsigned BAR_ABORT = 0x80000000u;     // set in the barrier word by a block that gave up
constexpr unsigned long long BAR_WAIT_NS = 1000000000ull;  // a barrier wait gives up after 1 s

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier: the barrier word counts arrivals; barrier number k is passed
// once it reaches (k + 1) * gridDim.x.  A wait that lasts longer than BAR_WAIT_NS,
// or that sees another block's abort mark, records PDE_BARRIER, marks the word
// and returns false; every block then leaves the kernel.
__device__ bool grid_barrier(unsigned *bar, unsigned target, unsigned *err, int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned long long t0 = global_ns();
        for (unsigned it = 1;; ++it) {
            const unsigned v = ld_acquire_u32(bar);
            if (v & BAR_ABORT) { ok = 0; break; }
            if (v >= target) break;
            if ((it & 63u) == 0 && global_ns() - t0 > BAR_WAIT_NS) {
                atomicOr(err, (unsigned)PDE_BARRIER);
                atomicOr(bar, BAR_ABORT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// The wall reactions of one step from the per-block partials (the last-block
// reduction of block_finish: one warp per component, lanes striding over the
// blocks, a fixed xor butterfly), written with the impulse by block 0.
__device__ __forceinline__ void reduce_reactions(const StepParams &p, const double *partials, int nblocks)
{
    const int ncomp = 3 * p.walls.nw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = warp; c < ncomp; c += STEP_THREADS / 32) {
        double s = 0.0;
#pragma unroll 8
        for (int b = lane; b < nblocks; b += 32) s += __ldcg(partials + (int64_t)b * PART_STRIDE + c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            p.react[c] = s;
            p.impulse[c] = dadd(p.impulse[c], dmul(p.dt, s));
        }
    }
}

template <int G, bool MIXED, bool WX>
__device__ __forceinline__ bool persist_step(const StepParams &p, int step, unsigned *bar, unsigned &nbar, unsigned arrivals,
                                             double (*s_react)[PD_MAX_WALLS * 3], double *s_vmax, double *s_wall,
                                             unsigned &s_err, int &s_ok, double &s_disp)
{
    constexpr int GPB = STEP_THREADS / G;
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    if (p.pair_diss && p.contact && p.cand_fd) {  // damping and friction of the candidates first
        pair_damping_rows<MIXED>(p, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
        if (!grid_barrier(bar, ++nbar * arrivals, p.err, &s_ok)) return false;
    }
    if (gl == 0)
        for (int q = 0; q < PD_MAX_WALLS * 3; ++q) s_react[grp][q] = 0.0;
    if (threadIdx.x == 0) s_err = 0;
    __syncthreads();
    unsigned err = 0;
    double vmax2 = 0.0;
    float vmax2f = 0.f;
    const TileView tv{nullptr, nullptr, nullptr, false};
    for (int64_t r0 = (int64_t)blockIdx.x * GPB; r0 < p.n; r0 += (int64_t)gridDim.x * GPB) {
        const int64_t row = r0 + grp;
        process_row<G, MIXED, WX, false>(p, s_wall, row, row < p.n, gl, 0, tv, s_react[grp], err, vmax2f, vmax2);
    }
    if (gl == 0) s_vmax[grp] = MIXED ? (double)vmax2f : vmax2;
    if (err) atomicOr(&s_err, err);
    __syncthreads();
    // this block's partials, in the buffer of the step's parity
    double *partials = p.partials + (int64_t)(step & 1) * gridDim.x * PART_STRIDE;
    double *part = partials + (int64_t)blockIdx.x * PART_STRIDE;
    const int ncomp = 3 * p.walls.nw;
    if ((int)threadIdx.x < ncomp) {
        double sum = 0.0;
        for (int g = 0; g < GPB; ++g) sum += s_react[g][threadIdx.x];
        part[threadIdx.x] = sum;
    } else if (threadIdx.x == 32) {
        double m = 0.0;
        for (int g = 0; g < GPB; ++g) m = fmax(m, s_vmax[g]);
        part[PART_STRIDE - 2] = m > 0.0 ? (double)__double2float_ru(m) : 0.0;
        if (s_err) atomicOr(p.err, s_err);
    }
    if (!grid_barrier(bar, ++nbar * arrivals, p.err, &s_ok)) return false;
    if (blockIdx.x == 0) reduce_reactions(p, partials, gridDim.x);
    {  // the same bookkeeping in every block: max |v|^2 over the blocks' partials,
       // read by all threads at once (a max does not depend on the order)
        double vm = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += STEP_THREADS)
            vm = fmax(vm, __ldcg(partials + (int64_t)b * PART_STRIDE + PART_STRIDE - 2));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vm = fmax(vm, __shfl_xor_sync(0xffffffffu, vm, o));
        if ((threadIdx.x & 31) == 0) s_vmax[threadIdx.x >> 5] = vm;  // s_vmax holds >= 8 entries (G <= 32)
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = 0.0;
            for (int w = 0; w < STEP_THREADS / 32; ++w) m = fmax(m, s_vmax[w]);
            s_disp = s_disp + p.dt * sqrt(m);
        }
    }
    if ((int)threadIdx.x < ncomp) {
        const int l = threadIdx.x / 3, q = threadIdx.x % 3;
        s_wall[threadIdx.x] = dadd(s_wall[threadIdx.x], dmul(p.dt, p.walls.v[l][q]));
    }
    __syncthreads();
    return true;
}

template <int G, bool MIXED, bool WX>
__global__ void __launch_bounds__(STEP_THREADS, 2)
    k_persist(const __grid_constant__ StepParams pa, const __grid_constant__ StepParams pb, int nsteps, unsigned *bar,
              unsigned absent)
{
    // a barrier is passed once every block has arrived; `absent` (0 in use) adds
    // arrivals that never come, which tests the bounded wait and its error status
    const unsigned arrivals = gridDim.x + absent;
    constexpr int GPB = STEP_THREADS / G;
    __shared__ double s_react[GPB][PD_MAX_WALLS * 3];
    __shared__ double s_vmax[GPB];
    __shared__ double s_wall[PD_MAX_WALLS * 3];
    __shared__ unsigned s_err;
    __shared__ int s_ok;
    __shared__ double s_disp;
    const int ncomp = 3 * pa.walls.nw;
    if ((int)threadIdx.x < ncomp) s_wall[threadIdx.x] = pa.wall_pos[threadIdx.x];
    if (threadIdx.x == 0) {
        s_disp = *pa.disp;
        if (blockIdx.x == 0 && pa.contact && *pa.stale) atomicOr(pa.err, (unsigned)PDE_SKIN);
    }
    __syncthreads();
    unsigned nbar = 0;
    int done = 0;
    for (int st = 0; st < nsteps; ++st) {
        // a list that went stale in the previous step of this run: the next step
        // would use it, so the run stops here with the stale mark (as k_step does)
        if (st > 0 && pa.contact && 2.0 * s_disp >= pa.skin) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(pa.err, (unsigned)PDE_SKIN);
            break;
        }
        // one copy of the step's code for both parities: the parameter block is
        // chosen at run time (grid-constant parameters can be addressed)
        const StepParams &p = (st & 1) ? pb : pa;
        const bool ok =
            persist_step<G, MIXED, WX>(p, st, bar, nbar, arrivals, s_react, s_vmax, s_wall, s_err, s_ok, s_disp);
        if (!ok) return;
        done = st + 1;
    }
    if (blockIdx.x == 0) {
        if ((int)threadIdx.x < ncomp) pa.wall_pos[threadIdx.x] = s_wall[threadIdx.x];
        if (threadIdx.x == 0 && done > 0) {
            *pa.disp = s_disp;
            if (2.0 * s_disp >= pa.skin) *pa.stale = 1;
        }
    }
}

// Mixed path with shared-memory tiles.  A block takes tile t (rows
// [t T, (t+1) T)) and stages in shared memory everything its rows read: row
// pointers, the tile's slice of 16-bit local neighbour indices (bit 15 = broken),
// the records of the tile's node list, and the rows' velocities.  The bond loop
// then makes no global loads.  Tiles whose list exceeds the capacity take the
// global-gather path of process_row.
template <int G>
__global__ void __launch_bounds__(STEP_THREADS, PD_MINB_TILED) k_step_tiled(const StepParams p)
{
    constexpr int GPB = STEP_THREADS / G;
    extern __shared__ float4 s_rec[];
    __shared__ double s_react[GPB][PD_MAX_WALLS * 3];
    __shared__ double s_vmax[GPB];
    __shared__ unsigned s_err;
    __shared__ bool s_last;
    const int T = p.tile_rows, cap = p.tile_cap;
    float4 *r0s = s_rec, *r1s = r0s + cap, *r2s = r1s + cap, *vhs = r2s + cap, *vls = vhs + T;
    // row pointers: T + 1 entries, padded to an even count so that the 16-bit
    // arrays after them (filled with 16-byte stores) start 16-byte aligned
    int64_t *rps = (int64_t *)(vls + T);
    uint16_t *lrs = (uint16_t *)(rps + ((T + 2) & ~1));
    uint16_t *lcs = lrs + ((T + 7) & ~7);
    const int gl = threadIdx.x % G, grp = threadIdx.x / G;
    if (gl == 0) {
        for (int q = 0; q < PD_MAX_WALLS * 3; ++q) s_react[grp][q] = 0.0;
    }
    if (threadIdx.x == 0) {
        s_err = 0;
        if (blockIdx.x == 0 && p.contact && *p.stale) atomicOr(p.err, (unsigned)PDE_SKIN);
    }
    if (segment_doomed(p)) return;  // uniform over the grid (see segment_doomed)
    __syncthreads();
    unsigned err = 0;
    double vmax2 = 0.0;
    float vmax2f = 0.f;
    const TileView off{nullptr, nullptr, nullptr, false};
    for (int64_t t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
        const int64_t base = p.tile_ptr[t];
        const int len = (int)(p.tile_ptr[t + 1] - base);
        const int64_t r0 = t * T;
        const int rows = (int)min((int64_t)T, p.n - r0);
        const bool on = len <= cap;
        int64_t ka = 0;
        if (on) {
            const int64_t kbase = __ldg(p.rowptr + r0), kend = __ldg(p.rowptr + r0 + rows);
            ka = kbase & ~(int64_t)7;  // 16-byte aligned start of the index slice
            const int nch = (int)((kend - ka + 7) >> 3);
            const uint4 *src = (const uint4 *)(p.lcol + ka);
            for (int q = threadIdx.x; q < nch; q += STEP_THREADS) ((uint4 *)lcs)[q] = src[q];
            for (int q = threadIdx.x; q <= rows; q += STEP_THREADS) rps[q] = __ldg(p.rowptr + r0 + q);
            for (int q = threadIdx.x; q < rows; q += STEP_THREADS) {
                vhs[q] = p.vh[r0 + q];
                vls[q] = p.vl[r0 + q];
                lrs[q] = __ldg(p.lrow + r0 + q);
            }
            for (int q = threadIdx.x; q < len; q += STEP_THREADS) {
                const int j = __ldg(p.ulist + base + q);
                r0s[q] = __ldg(p.xh4 + RECX * j);
                r1s[q] = __ldg(p.uh_in + REC * j);
                r2s[q] = __ldg(p.ul_in + REC * j);
            }
        }
        __syncthreads();
        for (int rr = grp; rr < T; rr += GPB) {
            const int64_t row = r0 + rr;
            const bool active = rr < rows;
            if (!on) {
                process_row<G, true>(p, p.wall_pos, row, active, gl, 0, off, s_react[grp], err, vmax2f, vmax2);
                continue;
            }
            float fbx = 0.f, fby = 0.f, fbz = 0.f;
            float4 o0, o1, o2;
            if (active) {
                const int lr = lrs[rr];
                o0 = r0s[lr]; o1 = r1s[lr]; o2 = r2s[lr];
                float ol[3];
                xl_unpack(o1.w, o2.w, ol);
                const int i0 = (int)rps[rr], i1 = (int)rps[rr + 1], kofs = (int)ka;
                for (int k = i0 + gl; k < i1; k += PD_INFLIGHT * G) {
                    uint32_t ll[PD_INFLIGHT];
#pragma unroll
                    for (int q = 0; q < PD_INFLIGHT; ++q) {
                        const int kq = k + q * G;
                        ll[q] = kq < i1 ? lcs[kq - kofs] : 0x8000u;
                    }
                    float4 a0[PD_INFLIGHT], a1[PD_INFLIGHT], a2[PD_INFLIGHT];
#pragma unroll
                    for (int q = 0; q < PD_INFLIGHT; ++q) {
                        const uint32_t iq = ll[q] & 0x7fffu;
                        a0[q] = r0s[iq]; a1[q] = r1s[iq]; a2[q] = r2s[iq];
                    }
#pragma unroll
                    for (int q = 0; q < PD_INFLIGHT; ++q)
                        if (!(ll[q] & 0x8000u))
                            bond_mixed<true>(p, k + q * G, o0, o1, o2, ol, a0[q], a1[q], a2[q], fbx, fby, fbz);
                }
            }
            __syncwarp();
            // contact candidates (rare; FP64 from global memory, ordered sum)
            double cx, cy, cz;
            contact_sum<G, true>(p, row, active, gl, cx, cy, cz);
            fbx = group_sum<G>(fbx) + (float)cx;
            fby = group_sum<G>(fby) + (float)cy;
            fbz = group_sum<G>(fbz) + (float)cz;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            err |= epilogue_lanes<G, false>(p, p.wall_pos, row, active, gl, fbx, fby, fbz, active ? o0 : z4, active ? o1 : z4,
                                     active ? o2 : z4, active ? vhs[rr] : z4, active ? vls[rr] : z4, s_react[grp],
                                     vmax2f);
        }
        __syncthreads();
    }
    if (gl == 0) s_vmax[grp] = (double)vmax2f;
    block_finish<GPB>(p, s_react, s_vmax, s_err, s_last, err);
}

// First half of a chunk's first step: v += dt/2 a; u^{n+1} = u^n + dt v; walls move.
// The drift's displacement bound (dt times the largest |v|) enters the contact
// list's bookkeeping as every fused step's drift does, by the last block: a list
// carried over from the previous call is checked against it before the forces use
// it (the rebuild that follows a drift otherwise resets it).  256 threads a block.
template <bool MIXED>
__global__ void k_drift(const StepParams p)
{
    __shared__ float s_m[8];
    __shared__ bool s_last;
    const double hdt = 0.5 * p.dt;
    float vm = 0.f;  // largest |v|^2 after the half kick (FP32, as the fused steps keep it)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (MIXED) {
            const float4 a = p.af[i], vh = p.vh[i], vl = p.vl[i], uh = p.uh_in[REC * i], ul = p.ul_in[REC * i];
            const df h{p.hdt_hi, p.hdt_lo}, dt{p.dt_hi, p.dt_lo};
            const df vx = df_on_fp64_grid(df_add(df{vh.x, vl.x}, df_mul_f(h, a.x)));
            const df vy = df_on_fp64_grid(df_add(df{vh.y, vl.y}, df_mul_f(h, a.y)));
            const df vz = df_on_fp64_grid(df_add(df{vh.z, vl.z}, df_mul_f(h, a.z)));
            const df ux = df_on_fp64_grid(df_add(df{uh.x, ul.x}, df_mul(dt, vx)));
            const df uy = df_on_fp64_grid(df_add(df{uh.y, ul.y}, df_mul(dt, vy)));
            const df uz = df_on_fp64_grid(df_add(df{uh.z, ul.z}, df_mul(dt, vz)));
            p.vh[i] = make_float4(vx.hi, vy.hi, vz.hi, 0.f);
            p.vl[i] = make_float4(vx.lo, vy.lo, vz.lo, 0.f);
            p.uh_out[REC * i] = make_float4(ux.hi, uy.hi, uz.hi, uh.w);
            p.ul_out[REC * i] = make_float4(ux.lo, uy.lo, uz.lo, ul.w);
            vm = fmaxf(vm, vx.hi * vx.hi + vy.hi * vy.hi + vz.hi * vz.hi);
        } else {
            dbl4 v = p.v[i];
            const dbl4 a = p.acc[i], u = p.u_in[i];
            v.x = dadd(v.x, dmul(hdt, a.x));
            v.y = dadd(v.y, dmul(hdt, a.y));
            v.z = dadd(v.z, dmul(hdt, a.z));
            dbl4 un;
            un.x = dadd(u.x, dmul(p.dt, v.x));
            un.y = dadd(u.y, dmul(p.dt, v.y));
            un.z = dadd(u.z, dmul(p.dt, v.z));
            un.w = 0.0;
            p.v[i] = v;
            p.u_out[i] = un;
            vm = fmaxf(vm, __double2float_ru(v.x * v.x + v.y * v.y + v.z * v.z));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int l = 0; l < p.walls.nw; ++l)
            for (int q = 0; q < 3; ++q)
                p.wall_pos[3 * l + q] = dadd(p.wall_pos[3 * l + q], dmul(p.dt, p.walls.v[l][q]));
    }
    if (!p.contact) return;  // uniform: a kernel parameter
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = vm;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < 8; ++w) m = fmaxf(m, s_m[w]);
        if (m > 0.f) atomicMax(p.vmax_bits, __float_as_uint(m));  // non-negative floats order as their bits
        __threadfence();
        s_last = atomicAdd(p.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const double m = (double)__uint_as_float(atomicExch(p.vmax_bits, 0u));
        const double dsp = *p.disp + p.dt * sqrt(m);
        *p.disp = dsp;
        if (2.0 * dsp >= p.skin) *p.stale = 1;
        *p.counter = 0u;
    }
}

// u (FP64) from the double-float state, for the rebuild kernels and queries
__global__ void k_materialize(const float4 *__restrict__ hi, const float4 *__restrict__ lo, int stride, int64_t n,
                              dbl4 *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 h = hi[stride * i], l = lo[stride * i];
        dbl4 r;
        r.x = df_to_double(df{h.x, l.x});
        r.y = df_to_double(df{h.y, l.y});
        r.z = df_to_double(df{h.z, l.z});
        r.w = 0.0;
        out[i] = r;
    }
}

// double -> double-float; with xl (the static x_lo) the spare lanes get the packed
// x_lo of the u records
__global__ void k_split_df(const dbl4 *__restrict__ in, const float4 *__restrict__ xl, int64_t n, float4 *hi,
                           float4 *lo, int stride)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const dbl4 a = in[i];
        const df x = df_from_double(a.x), y = df_from_double(a.y), z = df_from_double(a.z);
        float w1 = 0.f, w2 = 0.f;
        if (xl) {
            const float4 q = xl[i];
            const uint32_t bx = __bfloat16_as_ushort(__float2bfloat16_rn(q.x));
            const uint32_t by = __bfloat16_as_ushort(__float2bfloat16_rn(q.y));
            const uint32_t bz = __bfloat16_as_ushort(__float2bfloat16_rn(q.z));
            w1 = __uint_as_float(bx | (by << 16));
            w2 = __uint_as_float(bz);
        }
        hi[stride * i] = make_float4(x.hi, y.hi, z.hi, w1);
        lo[stride * i] = make_float4(x.lo, y.lo, z.lo, w2);
    }
}

// x slot of the records: (x_hi, c V) with c the micromodulus as FP32 (the bond
// force uses V only as c V)
__global__ void k_fill_record_x(const float4 *__restrict__ xh4, int64_t n, float cf, float4 *rec)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float4 r = xh4[i];
        r.w = cf * r.w;
        rec[RECX * i] = r;
    }
}

template <int G>
void launch_g(const StepParams &p, int blocks, cudaStream_t st, bool mixed)
{
    if (p.wall_extra) {  // contexts with wall extras never take the tiled path
        if (mixed)
            k_step<G, true, true><<<blocks, STEP_THREADS, 0, st>>>(p);
        else
            k_step<G, false, true><<<blocks, STEP_THREADS, 0, st>>>(p);
    } else if (mixed && p.pairs) {  // each bond once: pass 1, then pass 2 with the update
        k_pairs_upper<G><<<blocks, STEP_THREADS, 0, st>>>(p);
        k_step<G, true, false, true><<<blocks, STEP_THREADS, 0, st>>>(p);
    } else if (mixed && p.tile_cap > 0) {
        const size_t smem = tiled_smem(p.tile_cap, p.tile_rows, p.tile_slot_cap);
        k_step_tiled<G><<<blocks, STEP_THREADS, smem, st>>>(p);
    } else if (mixed) {
        k_step<G, true, false><<<blocks, STEP_THREADS, 0, st>>>(p);
    } else {
        k_step<G, false, false><<<blocks, STEP_THREADS, 0, st>>>(p);
    }
}

template <int G>
cudaError_t launch_persist_g(const StepParams &pa, const StepParams &pb, int nsteps, int blocks, unsigned *bar,
                             unsigned absent, bool mixed, cudaStream_t st)
{
    void *args[] = {(void *)&pa, (void *)&pb, (void *)&nsteps, (void *)&bar, (void *)&absent};
    const void *fn;
    if (pa.wall_extra)
        fn = mixed ? (const void *)k_persist<G, true, true> : (const void *)k_persist<G, false, true>;
    else
        fn = mixed ? (const void *)k_persist<G, true, false> : (const void *)k_persist<G, false, false>;
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(STEP_THREADS), args, 0, st);
}

template <int G>
int persist_blocks_g(int sms, bool mixed, bool wx)
{
    int per = 0;
    const void *fn = wx ? (mixed ? (const void *)k_persist<G, true, true> : (const void *)k_persist<G, false, true>)
                        : (mixed ? (const void *)k_persist<G, true, false> : (const void *)k_persist<G, false, false>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, STEP_THREADS, 0);
    return sms * per;
}

template <int G>
int blocks_g(int sms, bool mixed, bool tiled, size_t smem)
{
    int per = 0;
    if (mixed && tiled) {
        cudaFuncSetAttribute(k_step_tiled<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_tiled<G>, STEP_THREADS, smem);
    } else if (mixed) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step<G, true, false>, STEP_THREADS, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step<G, false, false>, STEP_THREADS, 0);
    }
    if (per < 1) per = 1;
    return sms * per;
}

}  // namespace

// bytes of dynamic shared memory of k_step_tiled
size_t tiled_smem(int tile_cap, int tile_rows, int slot_cap)
{
    return (size_t)(3 * tile_cap + 2 * tile_rows) * sizeof(float4) + (size_t)((tile_rows + 2) & ~1) * sizeof(int64_t) +
           (size_t)((tile_rows + 7) & ~7) * 2 + (size_t)(slot_cap + 16) * 2;
}

// Grid of the step kernel: SMs x resident blocks per SM (persistent loops).
int step_blocks(int lanes, int device, bool mixed, bool tiled, size_t tile_smem)
{
    const size_t tile_cap = tile_smem;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (sms < 1) sms = 1;
    switch (lanes) {
        case 4: return blocks_g<4>(sms, mixed, tiled, tile_cap);
        case 8: return blocks_g<8>(sms, mixed, tiled, tile_cap);
        case 16: return blocks_g<16>(sms, mixed, tiled, tile_cap);
        default: return blocks_g<32>(sms, mixed, tiled, tile_cap);
    }
}

// Most blocks a cooperative launch of the multi-step kernel may have (0: none).
int persist_blocks(int lanes, int device, bool mixed, bool wx)
{
    int sms = 0, coop = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (sms < 1 || !coop) return 0;
    switch (lanes) {
        case 4: return persist_blocks_g<4>(sms, mixed, wx);
        case 8: return persist_blocks_g<8>(sms, mixed, wx);
        case 16: return persist_blocks_g<16>(sms, mixed, wx);
        default: return persist_blocks_g<32>(sms, mixed, wx);
    }
}

// nsteps MODE_FULL steps in one cooperative launch; pa for even steps, pb for odd
// ones.  bar (one word) must be zero.  Returns the launch status.
cudaError_t launch_persist(const StepParams &pa, const StepParams &pb, int nsteps, int lanes, int blocks,
                           unsigned *bar, unsigned absent, cudaStream_t st)
{
    const bool mixed = pa.xh4 != nullptr;
    switch (lanes) {
        case 4: return launch_persist_g<4>(pa, pb, nsteps, blocks, bar, absent, mixed, st);
        case 8: return launch_persist_g<8>(pa, pb, nsteps, blocks, bar, absent, mixed, st);
        case 16: return launch_persist_g<16>(pa, pb, nsteps, blocks, bar, absent, mixed, st);
        default: return launch_persist_g<32>(pa, pb, nsteps, blocks, bar, absent, mixed, st);
    }
}

void launch_step(const StepParams &p, int lanes, int blocks, cudaStream_t st)
{
    const bool mixed = p.xh4 != nullptr;
    if (p.pair_diss && p.contact && p.cand_fd) {
        const int db = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (p.n + 127) / 128));
        if (mixed)
            k_pair_damping<true><<<db, 128, 0, st>>>(p);
        else
            k_pair_damping<false><<<db, 128, 0, st>>>(p);
    }
    switch (lanes) {
        case 4: launch_g<4>(p, blocks, st, mixed); break;
        case 8: launch_g<8>(p, blocks, st, mixed); break;
        case 16: launch_g<16>(p, blocks, st, mixed); break;
        default: launch_g<32>(p, blocks, st, mixed); break;
    }
}

static int small_grid(int64_t n)
{
    int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

void materialize_df(const float4 *hi, const float4 *lo, int stride, int64_t n, dbl4 *out, cudaStream_t st)
{
    k_materialize<<<small_grid(n), 256, 0, st>>>(hi, lo, stride, n, out);
}

void split_df(const dbl4 *in, const float4 *xl, int64_t n, float4 *hi, float4 *lo, int stride, cudaStream_t st)
{
    k_split_df<<<small_grid(n), 256, 0, st>>>(in, xl, n, hi, lo, stride);
}

void fill_record_x(const float4 *xh4, int64_t n, float cf, float4 *rec, cudaStream_t st)
{
    k_fill_record_x<<<small_grid(n), 256, 0, st>>>(xh4, n, cf, rec);
}

void launch_drift(const StepParams &p, cudaStream_t st)
{
    int blocks = (int)((p.n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (p.xh4)
        k_drift<true><<<blocks, 256, 0, st>>>(p);
    else
        k_drift<false><<<blocks, 256, 0, st>>>(p);
}
