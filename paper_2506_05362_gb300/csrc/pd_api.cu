// C ABI of libpd: context management, set-up, CUDA-graph stepping, queries.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pd_build.cuh"
#include "pd_grid.cuh"
#include "pd_internal.cuh"

// the multi-step kernel is the default up to this many nodes
#ifndef PD_PERSIST_AUTO_NODES
#define PD_PERSIST_AUTO_NODES 20000
#endif

struct GraphEntry {
    int steps, k, parity;
    bool skip0;  // no contact-list rebuild before the first step
    double dt;
    cudaGraphExec_t exec;
    int64_t launches;
};

struct pd_ctx {
    pd_options opt;
    pd_material mat;
    cudaStream_t st = nullptr;
    std::string err;
    std::vector<void *> owned;

    int64_t n = 0;
    double lo[3], hi[3];
    double K = 0, c = 0, s0 = 0, Kn = 0, delta = 0;
    bool bonds_ready = false;
    int64_t B = 0;
    int sh = 1;  // bits per node index

    int32_t *perm = nullptr, *inv = nullptr, *grain = nullptr;
    dbl4 *x4 = nullptr, *u[2] = {nullptr, nullptr}, *v = nullptr, *acc = nullptr, *F = nullptr;
    float4 *xh4 = nullptr, *xl4 = nullptr;
    float4 *rec[2] = {nullptr, nullptr};                 // mixed path: node record buffers (rec_float4s(n) float4), current / next
    float4 *uh[2] = {nullptr, nullptr}, *ul[2] = {nullptr, nullptr};  // views of the u slots (stride REC)
    float4 *vh = nullptr, *vl = nullptr, *af = nullptr;  // mixed path: v pairs, a
    float4 *snap_vh = nullptr, *snap_vl = nullptr, *snap_af = nullptr, *snap_rec = nullptr;
    bool own_stream = false;
    int cur = 0;

    int64_t *rowptr = nullptr, *crow = nullptr;
    int32_t *col = nullptr, *kc_of = nullptr;
    uint32_t *brk = nullptr;
    int64_t nwords = 0;

    // contact candidates and grid
    int64_t *cand_ptr = nullptr, *cand_cnt = nullptr;
    int2 *cand = nullptr;
    int64_t cand_cap = 0;
    dbl4 *cand_fd = nullptr;  // pair damping + friction force per candidate (float4 view on the mixed path)
    double fric_dt = 0;       // time step the friction's stick branch sees (that of the latest pd_step)
    double *gl = nullptr;     // Gauss-Legendre table of the multi-wall overlap terms
    uint32_t *gk = nullptr, *gk2 = nullptr, *gv = nullptr, *gv2 = nullptr, *gstart = nullptr, *gend = nullptr;
    uint64_t *gcell = nullptr;
    float4 *gpf = nullptr;  // FP32 positions of the grid's nodes (distance prefilter)
    uint32_t nbuckets = 0;
    int64_t *tmp = nullptr;  // scan / radix scratch for n-sized problems

    // reductions and device scalars
    double *partials = nullptr, *react = nullptr, *disp = nullptr, *wall_pos = nullptr, *dscratch = nullptr;
    unsigned *counter = nullptr, *derr = nullptr, *vmax_bits = nullptr, *dflag = nullptr;
    int *stale = nullptr;
    int blocks = 0, lanes = 0, blocks_cap = 0;
    double tune_ms[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // global, tiled, each bond once; 4/8/16/32 lanes
    // shared-memory tiles of the mixed path
    int64_t *tile_ptr = nullptr;
    int32_t *ulist = nullptr;
    uint16_t *lcol = nullptr, *lrow = nullptr;
    int32_t *colf = nullptr;  // col with the broken flag in bit 31 (mixed path; bitset is the master)
    int64_t ntiles = 0;
    int tile_rows = 64, tile_cap = 0, tile_slot_cap = 0;
    size_t tile_smem = 0;
    bool tiled = false;
    // each bond once (mixed path): split, mirror slots, per-slot factors, pass 1's row forces
    int32_t *split = nullptr, *mir = nullptr;
    float *tb = nullptr;
    float4 *fup = nullptr;
    bool pairs_ok = false, pairs = false;
    // several steps per launch (cooperative multi-step kernel of the global kernels)
    unsigned *gbar = nullptr;
    bool persist = false;
    cudaError_t launch_err = cudaSuccess;
    double centre[3] = {0, 0, 0};

    WallSet walls;
    double b[3] = {0, 0, 0};
    double t = 0;
    unsigned latched = 0;

    // staging and snapshot
    double *stage = nullptr;   // n*3 doubles
    uint8_t *stage_b = nullptr;  // B bytes
    dbl4 *snap_u = nullptr, *snap_v = nullptr, *snap_acc = nullptr;
    uint32_t *snap_brk = nullptr;
    uint32_t *stage_bits = nullptr;  // a caller's bond memory in internal order (pd_set_state*)
    int64_t n_state_applied = 0, n_state_unchanged = 0;  // pd_set_state* calls by outcome

    std::vector<GraphEntry> graphs;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double impulse_span = 0;       // time covered by the wall impulses since their reset
    int64_t n_rollbacks = 0, n_rebuilds = 0, n_steps = 0;  // since creation (successful segments' rebuilds)
    // the contact list on the device holds for the current state: built from it or
    // carried through steps whose displacement bound stayed inside the skin (the
    // device's stale flag clear); a one-step pd_step then needs no rebuild
    bool list_ok = false;
    int h_stale = 0;
    int k_cap = 1 << 30;  // rebuild period a stale list forced down; relaxed by 2x per clean segment
    double last_vm = 0;   // fastest speed at the previous segment's start
    double last_ms = 0, last_force_ms = 0;
    int64_t last_launches = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;  // pairs around force launches
    int prof_used = 0;
};

void *pd_dev_alloc(pd_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->opt.alloc) {
        p = c->opt.alloc(bytes, c->opt.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->owned.push_back(p);
    return p;
}

void pd_dev_free(pd_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find(c->owned.begin(), c->owned.end(), p);
    if (it != c->owned.end()) c->owned.erase(it);
    if (c->opt.free)
        c->opt.free(p, c->opt.alloc_ctx);
    else if (!c->opt.alloc)
        cudaFree(p);
}

namespace {

// n-point Gauss-Legendre rule mapped to [0, 1]: the roots of the Legendre
// polynomial P_n by Newton's method from the asymptotic first guesses
// cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' from the three-term recurrence;
// weight 2 / ((1 - z^2) P_n'(z)^2), halved for the unit interval.
void gauss_legendre01(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p2 = p1;
                p1 = p0;
                p0 = ((2 * j - 1) * z * p1 - (j - 1) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double z1 = z;
            z = z1 - p0 / dp;
            if (fabs(z - z1) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

pd_status fail(pd_ctx *c, pd_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            return fail(c, PD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
        }                                                                                         \
    } while (0)

#define ALLOC(ptr, type, count)                                                                   \
    do {                                                                                          \
        (ptr) = (type *)pd_dev_alloc(c, sizeof(type) * (size_t)(count));                          \
        if (!(ptr)) return fail(c, PD_ENOMEM, "device allocation failed: " #ptr);                 \
    } while (0)

template <typename T>
void release(pd_ctx *c, T *&p)
{
    pd_dev_free(c, (void *)p);
    p = nullptr;
}

void clear_graphs(pd_ctx *c)
{
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

int bits_for(int64_t v)
{
    int b = 1;
    while (b < 62 && ((int64_t)1 << b) <= v) ++b;
    return b;
}

pd_status sync(pd_ctx *c)
{
    CK(cudaStreamSynchronize(c->st));
    return PD_OK;
}

void constants(pd_ctx *c)
{
    const double nu = 0.25, E = c->mat.E, G0 = c->mat.G0, d = c->delta;
    c->K = E / (3.0 * (1.0 - 2.0 * nu));
    if (c->mat.micromodulus == 1 && c->mat.constants == 1) {  // conic, printed row
        c->c = 60.0 * E / (M_PI * pow(d, 5) * (1.0 - nu));
        c->s0 = sqrt(7.0 * M_PI * G0 / (12.0 * E * d));
    } else if (c->mat.micromodulus == 1) {  // conic: bulk and crack energies matched
        c->c = 90.0 * c->K / (M_PI * pow(d, 5));
        c->s0 = sqrt(2.0 * G0 / (3.0 * c->K * d));
    } else if (c->mat.constants == 1) {
        c->c = 12.0 * E / (M_PI * pow(d, 4) * (1.0 - nu));
        c->s0 = sqrt(5.0 * M_PI * G0 / (12.0 * E * d));
    } else {
        c->c = 18.0 * c->K / (M_PI * pow(d, 4));
        c->s0 = sqrt(5.0 * G0 / (9.0 * c->K * d));
    }
    c->Kn = c->mat.contact_factor * 18.0 * c->K / (M_PI * pow(d, 5));
}

double skin_of(const pd_ctx *c) { return c->opt.skin > 0 ? c->opt.skin : 0.5 * c->mat.contact_radius; }

StepParams params(pd_ctx *c, int mode, int in, double dt)
{
    StepParams p;
    memset(&p, 0, sizeof(p));
    const bool mixed = c->opt.precision == PD_MIXED;
    p.n = c->n;
    p.rowptr = c->rowptr;
    p.col = c->col;
    p.brk = c->brk;
    p.colf = c->colf;
    p.xh4 = mixed ? c->rec[in] : nullptr;
    p.xl4 = mixed ? c->xl4 : nullptr;
    p.uh_in = mixed ? c->uh[in] : nullptr;
    p.ul_in = mixed ? c->ul[in] : nullptr;
    p.uh_out = mixed ? c->uh[in ^ 1] : nullptr;
    p.ul_out = mixed ? c->ul[in ^ 1] : nullptr;
    p.vh = c->vh;
    p.vl = c->vl;
    p.af = c->af;
    {
        const float dth = (float)dt, hdth = (float)(0.5 * dt);
        p.dt_hi = dth;
        p.dt_lo = (float)(dt - (double)dth);
        p.hdt_hi = hdth;
        p.hdt_lo = (float)(0.5 * dt - (double)hdth);
        p.inv_rho_f = (float)(1.0 / c->mat.rho);
        for (int a = 0; a < 3; ++a) p.bf[a] = (float)c->b[a];
        p.Rc_f = (float)c->mat.contact_radius;
    }
    p.x4 = c->x4;
    p.u_in = c->u[in];
    p.u_out = c->u[in ^ 1];
    p.v = c->v;
    p.acc = c->acc;
    p.F_out = mode == MODE_FORCES ? c->F : nullptr;
    p.grain = c->grain;
    p.contact = c->opt.contact;
    p.cand_ptr = c->cand_ptr;
    p.cand = c->cand;
    p.c = c->c;
    p.s0 = c->s0;
    p.Kn = c->Kn;
    p.Rc = c->mat.contact_radius;
    p.rho = c->mat.rho;
    p.dt = dt;
    p.cf = (float)c->c;
    p.s0f = (float)c->s0;
    p.break_mode = c->mat.break_mode;
    p.beta_d = c->mat.beta_d;
    p.conic = c->mat.micromodulus == 1;
    p.delta = c->delta;
    p.delta_f = (float)c->delta;
    p.cand_fd = c->cand_fd;
    p.mu = c->mat.mu;
    p.dt_f = mode == MODE_FORCES ? c->fric_dt : dt;
    p.pair_diss = (c->mat.beta_d > 0 || c->mat.mu > 0) ? 1 : 0;
    p.wall_overlap = c->mat.wall_overlap;
    p.wall_extra = (c->walls.nw > 0 && (c->mat.mu > 0 || (c->mat.wall_overlap && c->walls.nw >= 2))) ? 1 : 0;
    p.wall_n = c->wall_pos + 2 * PD_MAX_WALLS * 3;
    p.gl = c->gl;
    p.mode = mode;
    p.walls = c->walls;
    p.wall_pos = c->wall_pos;
    for (int a = 0; a < 3; ++a) p.b[a] = c->b[a];
    p.partials = c->partials;
    p.counter = c->counter;
    p.vmax_bits = c->vmax_bits;
    p.err = c->derr;
    p.react = c->react;
    p.impulse = c->wall_pos + PD_MAX_WALLS * 3;
    p.disp = c->disp;
    p.skin = skin_of(c);
    p.stale = c->stale;
    for (int q = 0; q < 3; ++q) p.centre[q] = c->centre[q];
    if (mixed && c->pairs) {
        p.pairs = 1;
        p.split = c->split;
        p.mir = c->mir;
        p.tb = c->tb;
        p.fup = c->fup;
    } else if (mixed && c->tiled) {
        p.tile_cap = c->tile_cap;
        p.tile_slot_cap = c->tile_slot_cap;
        p.tile_rows = c->tile_rows;
        p.ntiles = c->ntiles;
        p.tile_ptr = c->tile_ptr;
        p.ulist = c->ulist;
        p.lcol = c->lcol;
        p.lrow = c->lrow;
    }
    return p;
}

// FP64 displacement of buffer `in` (materialised into scratch on the mixed path).
const dbl4 *upos(pd_ctx *c, int in)
{
    if (c->opt.precision == PD_MIXED) {
        materialize_df(c->uh[in], c->ul[in], REC, c->n, c->u[0], c->st);
        return c->u[0];
    }
    return c->u[in];
}

// Contact candidate rebuild from u[in] (stream-ordered; capturable).
void enqueue_rebuild(pd_ctx *c, int in)
{
    const dbl4 *u = upos(c, in);
    GridView g;
    for (int a = 0; a < 3; ++a) g.lo[a] = c->lo[a];
    const double cut = c->mat.contact_radius + skin_of(c);
    grid_build(g, c->x4, u, c->n, cut * (1.0 + 1e-7), c->nbuckets, c->gk, c->gk2, c->gv, c->gv2, c->gstart,
               c->gend, c->gcell, c->tmp, c->gpf, c->st);
    cand_count(c->x4, u, c->grain, c->rowptr, c->col, c->n, g, cut, c->cand_cnt, c->st);
    scan_exclusive_i64(c->cand_cnt, c->cand_ptr, c->n, c->tmp, c->st);
    cand_fill(c->x4, u, c->grain, c->rowptr, c->col, c->n, g, cut, c->cand_ptr, c->cand, c->cand_cap,
              c->derr, c->disp, c->stale, c->st);
}

pd_status grow_candidates(pd_ctx *c)
{
    int64_t need = 0;
    CK(cudaMemcpy(&need, c->cand_ptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    int64_t cap = std::max<int64_t>(2 * c->cand_cap, need + need / 2 + 1024);
    release(c, c->cand);
    ALLOC(c->cand, int2, cap);
    if (c->mat.beta_d > 0 || c->mat.mu > 0) {
        release(c, c->cand_fd);
        ALLOC(c->cand_fd, dbl4, cap);
    }
    c->cand_cap = cap;
    c->list_ok = false;
    clear_graphs(c);
    return PD_OK;
}

pd_status read_err(pd_ctx *c, unsigned *e)
{
    CK(cudaMemcpyAsync(e, c->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
    return PD_OK;
}

pd_status status_of(pd_ctx *c, unsigned e)
{
    if (e & PDE_NONFINITE) return fail(c, PD_ENONFINITE, "non-finite force or state on the device");
    if (e & PDE_WALL) return fail(c, PD_EWALL, "a node is a whole contact radius behind a wall");
    if (e & PDE_CAPACITY) return fail(c, PD_ECAPACITY, "contact candidate capacity exceeded");
    if (e & PDE_BARRIER) return fail(c, PD_ETIMEOUT, "a grid-wide barrier of the multi-step kernel timed out");
    if (e & PDE_SKIN) return fail(c, PD_ETIMEOUT, "contact list went stale between rebuilds");
    return PD_OK;
}

// Force evaluation at the current state (breaking applies).  Retries once after
// growing the candidate list.
// zero the wall impulses and the time they cover
cudaError_t reset_impulse(pd_ctx *c)
{
    c->impulse_span = 0;
    return cudaMemsetAsync(c->wall_pos + PD_MAX_WALLS * 3, 0, sizeof(double) * PD_MAX_WALLS * 3, c->st);
}

pd_status eval_forces(pd_ctx *c)
{
    for (int attempt = 0; attempt < 4; ++attempt) {
        if (c->opt.contact) enqueue_rebuild(c, c->cur);
        StepParams p = params(c, MODE_FORCES, c->cur, 0.0);
        launch_step(p, c->lanes, c->blocks, c->st);
        CK(cudaGetLastError());
        unsigned e = 0;
        pd_status s = read_err(c, &e);
        if (s) return s;
        if (e & PDE_CAPACITY) {
            s = grow_candidates(c);
            if (s) return s;
            continue;
        }
        e &= ~(unsigned)PDE_SKIN;
        c->latched |= e & (PDE_NONFINITE | PDE_WALL);
        c->list_ok = c->opt.contact != 0;  // rebuilt from this state just now
        return status_of(c, e);
    }
    return fail(c, PD_ECAPACITY, "contact candidate list could not be grown");
}

}  // namespace

// =============================================================================
extern "C" {

void pd_default_options(pd_options *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->device = 0;
    o->stream = nullptr;
    o->precision = PD_MIXED;
    o->contact = 1;
    o->contact_every = 0;
    o->skin = 0.0;
    o->lanes_per_node = 0;
    o->graph_chunk = 64;
}

const char *pd_last_error(const pd_ctx *c) { return c ? c->err.c_str() : "null context"; }

void pd_destroy(pd_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->opt.device);
    cudaStreamSynchronize(c->st);
    clear_graphs(c);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    std::vector<void *> own = c->owned;
    for (void *p : own) pd_dev_free(c, p);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

static pd_status create_impl(pd_ctx *c, const double *x, const double *vol, const int32_t *grain, const double *v0)
{
    const int64_t n = c->n;
    CK(cudaSetDevice(c->opt.device));
    c->st = (cudaStream_t)c->opt.stream;
    if (!c->st) {  // the legacy default stream cannot be captured into graphs
        CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    CK(cudaEventCreate(&c->ev0));
    CK(cudaEventCreate(&c->ev1));
    int32_t gmax = 0;
    for (int a = 0; a < 3; ++a) { c->lo[a] = INFINITY; c->hi[a] = -INFINITY; }
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double q = x[3 * i + a];
            if (!isfinite(q)) return fail(c, PD_EINVAL, "x contains a non-finite value");
            c->lo[a] = std::min(c->lo[a], q);
            c->hi[a] = std::max(c->hi[a], q);
        }
        if (!(vol[i] > 0) || !isfinite(vol[i])) return fail(c, PD_EINVAL, "vol must be positive and finite");
        if (grain[i] < 0) return fail(c, PD_EINVAL, "grain ids must be >= 0");
        gmax = std::max(gmax, grain[i]);
        if (v0)
            for (int a = 0; a < 3; ++a)
                if (!isfinite(v0[3 * i + a])) return fail(c, PD_EINVAL, "v0 contains a non-finite value");
    }
    c->sh = bits_for(n);
    // staging of the caller arrays
    double *dx, *dvol, *dv0 = nullptr;
    int32_t *dgrain;
    ALLOC(dx, double, 3 * n);
    ALLOC(dvol, double, n);
    ALLOC(dgrain, int32_t, n);
    CK(cudaMemcpyAsync(dx, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(dvol, vol, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(dgrain, grain, sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->st));
    if (v0) {
        ALLOC(dv0, double, 3 * n);
        CK(cudaMemcpyAsync(dv0, v0, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->st));
    }
    // scratch big enough for radix sorts and scans of n items
    int64_t tmpn = std::max(radix_tmp_size(n), scan_tmp_size(n + 1) + 8);
    ALLOC(c->tmp, int64_t, tmpn);
    uint64_t *k1, *k2;
    uint32_t *v1, *v2, *order;
    ALLOC(k1, uint64_t, n);
    ALLOC(k2, uint64_t, n);
    ALLOC(v1, uint32_t, n);
    ALLOC(v2, uint32_t, n);
    build_morton(dx, n, c->lo, c->hi, k1, k2, v1, v2, gmax > 0 ? bits_for(gmax) : 0, dgrain, c->tmp, &order, c->st);
    const bool mixed = c->opt.precision == PD_MIXED;
    ALLOC(c->perm, int32_t, n);
    ALLOC(c->inv, int32_t, n);
    ALLOC(c->grain, int32_t, n);
    ALLOC(c->x4, dbl4, n);
    ALLOC(c->v, dbl4, n);
    ALLOC(c->acc, dbl4, n);
    ALLOC(c->F, dbl4, n);
    for (int q = 0; q < 2; ++q) ALLOC(c->u[q], dbl4, n);
    if (mixed) {
        ALLOC(c->xh4, float4, n);
        ALLOC(c->xl4, float4, n);
        for (int q = 0; q < 2; ++q) {
            ALLOC(c->rec[q], float4, rec_float4s(n));
            c->uh[q] = c->rec[q] + rec_uh0(n);
            c->ul[q] = c->rec[q] + rec_ul0(n);
        }
        ALLOC(c->vh, float4, n);
        ALLOC(c->vl, float4, n);
        ALLOC(c->af, float4, n);
        ALLOC(c->snap_rec, float4, rec_float4s(n));
        ALLOC(c->snap_vh, float4, n);
        ALLOC(c->snap_vl, float4, n);
        ALLOC(c->snap_af, float4, n);
    }
    for (int q = 0; q < 3; ++q) c->centre[q] = 0.5 * (c->lo[q] + c->hi[q]);
    gather_nodes(order, n, dx, dvol, dgrain, dv0, c->perm, c->inv, c->x4, c->grain, c->v, c->xh4, c->xl4, c->centre,
                 c->st);
    CK(cudaGetLastError());
    for (int q = 0; q < 2; ++q) {
        CK(cudaMemsetAsync(c->u[q], 0, sizeof(dbl4) * n, c->st));
        if (mixed) CK(cudaMemsetAsync(c->rec[q], 0, sizeof(float4) * rec_float4s(n), c->st));
    }
    CK(cudaMemsetAsync(c->acc, 0, sizeof(dbl4) * n, c->st));
    CK(cudaMemsetAsync(c->F, 0, sizeof(dbl4) * n, c->st));
    if (mixed) {
        split_df(c->v, nullptr, n, c->vh, c->vl, 1, c->st);
        for (int q = 0; q < 2; ++q) {
            fill_record_x(c->xh4, n, 1.0f, c->rec[q], c->st);  // x slots are static (c V once bonds exist)
            split_df(c->u[q], c->xl4, n, c->uh[q], c->ul[q], REC, c->st);
        }
        CK(cudaMemsetAsync(c->af, 0, sizeof(float4) * n, c->st));
    }
    // grid and contact buffers
    uint32_t nb = 1024;
    while ((int64_t)nb < 2 * n && nb < (1u << 26)) nb <<= 1;
    c->nbuckets = nb;
    ALLOC(c->gk, uint32_t, n);
    ALLOC(c->gk2, uint32_t, n);
    ALLOC(c->gv, uint32_t, n);
    ALLOC(c->gv2, uint32_t, n);
    ALLOC(c->gstart, uint32_t, nb);
    ALLOC(c->gend, uint32_t, nb);
    ALLOC(c->gcell, uint64_t, n);
    ALLOC(c->gpf, float4, n);
    ALLOC(c->cand_ptr, int64_t, n + 1);
    ALLOC(c->cand_cnt, int64_t, n + 1);
    CK(cudaMemsetAsync(c->cand_ptr, 0, sizeof(int64_t) * (n + 1), c->st));
    c->cand_cap = c->opt.cand_capacity > 0 ? c->opt.cand_capacity : std::max<int64_t>(1024, 8 * n);
    ALLOC(c->cand, int2, c->cand_cap);
    if (c->mat.beta_d > 0 || c->mat.mu > 0) ALLOC(c->cand_fd, dbl4, c->cand_cap);  // damping + friction per candidate
    // reductions
    c->blocks_cap = 0;
    for (int g : {4, 8, 16, 32}) c->blocks_cap = std::max(c->blocks_cap, step_blocks(g, c->opt.device, mixed, false, 0));
    ALLOC(c->partials, double, 2 * (int64_t)c->blocks_cap * PART_STRIDE);  // two step parities (multi-step kernel)
    ALLOC(c->gbar, unsigned, 1);
    ALLOC(c->react, double, PD_MAX_WALLS * 3);
    ALLOC(c->disp, double, 1);
    ALLOC(c->wall_pos, double, PD_MAX_WALLS * 9);  // wall points, the wall impulses, the wall normals
    if (c->mat.wall_overlap) {
        double tab[2 * PD_GL];
        gauss_legendre01(PD_GL, tab, tab + PD_GL);
        ALLOC(c->gl, double, 2 * PD_GL);
        CK(cudaMemcpyAsync(c->gl, tab, sizeof(tab), cudaMemcpyHostToDevice, c->st));
    }
    ALLOC(c->dscratch, double, 8192);
    ALLOC(c->counter, unsigned, 1);
    ALLOC(c->vmax_bits, unsigned, 1);
    CK(cudaMemsetAsync(c->vmax_bits, 0, sizeof(unsigned), c->st));
    ALLOC(c->derr, unsigned, 1);
    ALLOC(c->dflag, unsigned, 1);
    ALLOC(c->stale, int, 1);
    CK(cudaMemsetAsync(c->react, 0, sizeof(double) * PD_MAX_WALLS * 3, c->st));
    CK(cudaMemsetAsync(c->disp, 0, sizeof(double), c->st));
    CK(cudaMemsetAsync(c->counter, 0, sizeof(unsigned), c->st));
    CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
    CK(cudaMemsetAsync(c->stale, 0, sizeof(int), c->st));
    ALLOC(c->stage, double, 6 * n);  // staging of u and v (pd_set_state checks both before applying)
    ALLOC(c->snap_u, dbl4, n);
    ALLOC(c->snap_v, dbl4, n);
    ALLOC(c->snap_acc, dbl4, n);
    c->walls.nw = 0;
    c->lanes = c->opt.lanes_per_node ? c->opt.lanes_per_node : 16;
    c->blocks = step_blocks(c->lanes, c->opt.device, mixed, false, 0);
    pd_status s = sync(c);
    if (s) return s;
    release(c, dx); release(c, dvol); release(c, dgrain); release(c, dv0);
    release(c, k1); release(c, k2); release(c, v1); release(c, v2);
    return PD_OK;
}

pd_status pd_create(int64_t n, const double *x, const double *vol, const int32_t *grain, const double *v0,
                    const pd_material *mat, const pd_options *opt, pd_ctx **out)
{
    if (!out) return PD_EINVAL;
    *out = nullptr;
    if (n < 1 || n > 0x7fffffffLL || !x || !vol || !grain || !mat) return PD_EINVAL;
    if (!(mat->E > 0) || !(mat->rho > 0) || !(mat->G0 > 0) || !(mat->contact_radius > 0) ||
        !(mat->contact_factor >= 0) || (mat->constants != 0 && mat->constants != 1) ||
        (mat->break_mode != 0 && mat->break_mode != 1) || !(mat->beta_d >= 0) || !isfinite(mat->beta_d) ||
        (mat->micromodulus != 0 && mat->micromodulus != 1) || !(mat->mu >= 0) || !isfinite(mat->mu) ||
        (mat->wall_overlap != 0 && mat->wall_overlap != 1))
        return PD_EINVAL;
    pd_ctx *c = new pd_ctx();
    if (opt) c->opt = *opt; else pd_default_options(&c->opt);
    if (c->opt.graph_chunk <= 0) c->opt.graph_chunk = 64;
    if (c->opt.precision != PD_MIXED && c->opt.precision != PD_FP64) { delete c; return PD_EINVAL; }
    int l = c->opt.lanes_per_node;
    if (l != 0 && l != 4 && l != 8 && l != 16 && l != 32) { delete c; return PD_EINVAL; }
    if (c->opt.tiles < -1 || c->opt.tiles > 1) { delete c; return PD_EINVAL; }
    if (c->opt.pairs < -1 || c->opt.pairs > 1 || (c->opt.pairs == 1 && c->opt.tiles == 1)) { delete c; return PD_EINVAL; }
    if (c->opt.persistent < -1 || c->opt.persistent > 1 || c->opt.barrier_absent < 0) { delete c; return PD_EINVAL; }
    if ((c->opt.alloc == nullptr) != (c->opt.free == nullptr)) { delete c; return PD_EINVAL; }
    if (c->opt.cand_capacity < 0) { delete c; return PD_EINVAL; }
    c->mat = *mat;
    c->n = n;
    pd_status s = create_impl(c, x, vol, grain, v0);
    if (s != PD_OK) {
        fprintf(stderr, "pd_create: %s\n", c->err.c_str());
        pd_destroy(c);
        return s;
    }
    *out = c;
    return PD_OK;
}

// Grid of the step kernel for `lanes` lanes per node: the resident blocks, but no
// more than the rows (or tiles) give work to (idle blocks only lengthen the
// fixed-order reduction of the wall reactions).
static int step_grid(const pd_ctx *c, int lanes)
{
    const bool mixed = c->opt.precision == PD_MIXED;
    const int64_t per = c->tiled ? c->tile_rows : 256 / lanes;
    const int64_t need = std::max<int64_t>(1, (c->n + per - 1) / per);
    const int b = std::min(c->blocks_cap, step_blocks(lanes, c->opt.device, mixed, c->tiled, c->tile_smem));
    return (int)std::min<int64_t>(b, need);
}

static pd_status autotune(pd_ctx *c)
{
    // time a force evaluation (idempotent at a fixed state) for each lane count and
    // each kernel the context can run: per-slot gathers from global memory (0),
    // shared-memory tiles (1), each bond once in two passes (2)
    const int cand[4] = {4, 8, 16, 32};
    const bool mixed = c->opt.precision == PD_MIXED;
    bool use[3] = {c->opt.tiles != 1 && c->opt.pairs != 1, c->tiled && c->opt.tiles != -1 && c->opt.pairs != 1,
                   c->pairs_ok && c->opt.pairs != -1 && c->opt.tiles != 1};
    if (!use[0] && !use[1] && !use[2]) use[0] = true;
    double best = INFINITY;
    int bestl = 16, bestk = 0;
    if (c->opt.contact) enqueue_rebuild(c, c->cur);
    for (int q = 0; q < 12; ++q) c->tune_ms[q] = 0;
    for (int q = 0; q < 4; ++q) {
        for (int kind = 0; kind < 3; ++kind) {
            if (!use[kind]) continue;
            const int l = cand[q];
            c->tiled = kind == 1;
            c->pairs = kind == 2;
            const int blocks = step_grid(c, l);
            StepParams p = params(c, MODE_FORCES, c->cur, 0.0);
            launch_step(p, l, blocks, c->st);  // warm-up; applies any breaking once
            CK(cudaEventRecord(c->ev0, c->st));
            for (int r = 0; r < 5; ++r) launch_step(p, l, blocks, c->st);
            CK(cudaEventRecord(c->ev1, c->st));
            CK(cudaEventSynchronize(c->ev1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
            const double t = ms / 5.0;
            c->tune_ms[4 * kind + q] = t;
            if (t < best) { best = t; bestl = l; bestk = kind; }
        }
    }
    // A full step adds per-node work to the force evaluation timed here (the Verlet
    // update on three lanes of each group, the grid rule of the state), which a
    // group of fewer lanes shares among more nodes per warp: of the winning kernel,
    // the fewest lanes within 3% of its best force evaluation are taken (on the
    // plate 4 and 8 lanes tie within 0.5% here, and 4 lanes are 4% faster a step).
    for (int q = 0; q < 4 && cand[q] < bestl; ++q) {
        const double t = c->tune_ms[4 * bestk + q];
        if (t > 0 && t <= 1.03 * best) { bestl = cand[q]; break; }
    }
    CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
    c->tiled = bestk == 1;
    c->pairs = bestk == 2;
    c->lanes = bestl;
    c->blocks = step_grid(c, bestl);
    clear_graphs(c);
    return sync(c);
}

pd_status pd_build_bonds(pd_ctx *c, double horizon, int nfilt, const pd_bond_filter *filt)
{
    if (!c) return PD_EINVAL;
    if (!(horizon > 0) || !isfinite(horizon) || nfilt < 0 || nfilt > PD_MAX_FILTERS || (nfilt > 0 && !filt))
        return fail(c, PD_EINVAL, "bad horizon or filter list");
    FilterSet f;
    memset(&f, 0, sizeof(f));
    f.nf = nfilt;
    for (int q = 0; q < nfilt; ++q) {
        if (filt[q].kind != 1 && filt[q].kind != 2) return fail(c, PD_EINVAL, "unknown filter kind");
        f.kind[q] = filt[q].kind;
        for (int a = 0; a < 12; ++a) f.a[q][a] = filt[q].a[a];
    }
    CK(cudaSetDevice(c->opt.device));
    clear_graphs(c);
    c->bonds_ready = false;
    release(c, c->rowptr); release(c, c->col); release(c, c->brk); release(c, c->kc_of);
    release(c, c->crow); release(c, c->snap_brk); release(c, c->stage_b); release(c, c->stage_bits);
    release(c, c->split); release(c, c->mir); release(c, c->tb); release(c, c->fup);
    c->pairs_ok = c->pairs = false;
    c->delta = horizon;
    constants(c);
    const int64_t n = c->n;
    if (c->opt.precision == PD_MIXED)  // the records carry c V for the bond force
        for (int q = 0; q < 2; ++q) fill_record_x(c->xh4, n, (float)c->c, c->rec[q], c->st);
    // grid over the reference positions, cell = horizon
    GridView g;
    for (int a = 0; a < 3; ++a) g.lo[a] = c->lo[a];
    grid_build(g, c->x4, nullptr, n, horizon * (1.0 + 1e-7), c->nbuckets, c->gk, c->gk2, c->gv, c->gv2, c->gstart,
               c->gend, c->gcell, c->tmp, c->gpf, c->st);
    int64_t *cnt;
    ALLOC(cnt, int64_t, n + 1);
    ALLOC(c->rowptr, int64_t, n + 1);
    bonds_count(c->x4, c->grain, c->perm, n, g, horizon, f, cnt, c->st);
    scan_exclusive_i64(cnt, c->rowptr, n, c->tmp, c->st);
    int64_t B = 0;
    CK(cudaMemcpyAsync(&B, c->rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
    pd_status s = sync(c);
    if (s) return s;
    if (B > 0x7fffffffLL) return fail(c, PD_ECAPACITY, "more than 2^31-1 directed bonds");
    c->B = B;
    uint64_t *k1, *k2;
    uint32_t *v1, *v2;
    int64_t *btmp;
    ALLOC(k1, uint64_t, B + 1);
    ALLOC(k2, uint64_t, B + 1);
    ALLOC(v1, uint32_t, B + 1);
    ALLOC(v2, uint32_t, B + 1);
    ALLOC(btmp, int64_t, std::max(radix_tmp_size(B + 1), scan_tmp_size(n + 1) + 8));
    ALLOC(c->col, int32_t, B + 1);
    bonds_fill(c->x4, c->grain, c->perm, n, g, horizon, f, c->rowptr, k1, c->sh, c->st);
    {
        uint64_t *k = k1, *ka = k2;
        radix_sort_u64(&k, &ka, nullptr, nullptr, B, 2 * c->sh, btmp, c->st);
        bonds_keys_to_col(k, B, c->sh, c->col, c->st);
    }
    // canonical numbering (caller rows, ascending caller columns)
    ALLOC(c->kc_of, int32_t, B + 1);
    ALLOC(c->crow, int64_t, n + 1);
    {
        canon_keys(c->rowptr, c->col, c->perm, n, c->sh, k1, v1, c->st);
        uint64_t *k = k1, *ka = k2;
        uint32_t *v = v1, *va = v2;
        radix_sort_u64(&k, &ka, &v, &va, B, 2 * c->sh, btmp, c->st);
        canon_invert(v, B, c->kc_of, c->st);
        row_len_caller(c->rowptr, c->inv, n, cnt, c->st);
        scan_exclusive_i64(cnt, c->crow, n, c->tmp, c->st);
    }
    // shared-memory tiles (mixed path): the largest tile (64, 32 or 16 rows) whose
    // staging fits two blocks per SM.  A material with friction or multi-wall terms
    // runs the global-gather kernels that carry the wall extras, so it has no tiles.
    release(c, c->tile_ptr); release(c, c->ulist); release(c, c->lcol); release(c, c->lrow);
    c->tiled = false;
    c->tile_cap = 0;
    if (c->opt.precision == PD_MIXED && c->opt.tiles >= 0 && !(c->mat.mu > 0) && !c->mat.wall_overlap) {
        const int64_t m = B + n;
        const size_t smem_max = 110 * 1024;
        std::vector<int64_t> rp(n + 1);
        CK(cudaMemcpyAsync(rp.data(), c->rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, c->st));
        uint64_t *tk1, *tk2;
        int64_t *flag, *pos, *ttmp;
        int32_t *ufull;
        ALLOC(tk1, uint64_t, m);
        ALLOC(tk2, uint64_t, m);
        ALLOC(flag, int64_t, m + 1);
        ALLOC(pos, int64_t, m + 1);
        ALLOC(ttmp, int64_t, std::max(radix_tmp_size(m), scan_tmp_size(m + 1) + 8));
        ALLOC(ufull, int32_t, m);
        ALLOC(c->lcol, uint16_t, B + 16);
        ALLOC(c->lrow, uint16_t, n);
        for (int T : {64, 32, 16}) {
            c->ntiles = (n + T - 1) / T;
            release(c, c->tile_ptr);
            ALLOC(c->tile_ptr, int64_t, c->ntiles + 1);
            const int cap_max = 32767;
            build_tiles(c->rowptr, c->col, n, B, T, c->sh, cap_max, tk1, tk2, flag, pos, ttmp, ufull, c->tile_ptr,
                        c->lcol, c->lrow, c->st);
            std::vector<int64_t> tp(c->ntiles + 1);
            CK(cudaMemcpyAsync(tp.data(), c->tile_ptr, sizeof(int64_t) * (c->ntiles + 1), cudaMemcpyDeviceToHost,
                               c->st));
            s = sync(c);
            if (s) return s;
            // capacity: the 99th-percentile list length (larger tiles gather globally)
            std::vector<int64_t> lens(c->ntiles);
            int64_t slot_cap = 0;
            for (int64_t t = 0; t < c->ntiles; ++t) {
                lens[t] = tp[t + 1] - tp[t];
                const int64_t r0 = t * T, r1 = std::min<int64_t>(n, r0 + T);
                slot_cap = std::max(slot_cap, rp[r1] - rp[r0]);
            }
            std::vector<int64_t> sorted = lens;
            std::sort(sorted.begin(), sorted.end());
            const int64_t cap = sorted[(size_t)((sorted.size() - 1) * 0.99)];
            const size_t smem = tiled_smem((int)cap, T, (int)slot_cap);
            if (smem <= smem_max || T == 16) {
                if (smem > smem_max) break;
                c->tile_rows = T;
                c->tile_cap = (int)cap;
                c->tile_slot_cap = (int)slot_cap;
                c->tile_smem = smem;
                const int64_t U = tp[c->ntiles];
                ALLOC(c->ulist, int32_t, U);
                CK(cudaMemcpyAsync(c->ulist, ufull, sizeof(int32_t) * U, cudaMemcpyDeviceToDevice, c->st));
                // local indices of tiles above the capacity are unused (global path)
                s = sync(c);
                if (s) return s;
                c->tiled = true;
                break;
            }
        }
        release(c, tk1); release(c, tk2); release(c, flag); release(c, pos); release(c, ttmp); release(c, ufull);
    }
    c->nwords = (B + 31) / 32 + 1;
    ALLOC(c->brk, uint32_t, c->nwords);
    ALLOC(c->snap_brk, uint32_t, c->nwords);
    ALLOC(c->stage_bits, uint32_t, c->nwords);
    ALLOC(c->stage_b, uint8_t, B + 16);
    CK(cudaMemsetAsync(c->brk, 0, sizeof(uint32_t) * c->nwords, c->st));
    // mixed path: neighbour index with the broken flag in bit 31, one word per slot
    release(c, c->colf);
    if (c->opt.precision == PD_MIXED) {
        ALLOC(c->colf, int32_t, B + 16);
        sync_colf_flags(c->brk, c->col, B, c->colf, c->st);
    }
    // each bond once (mixed path; materials whose walls need the extra terms run the
    // per-slot kernels that carry them)
    if (c->opt.precision == PD_MIXED && c->opt.pairs >= 0 && !(c->mat.mu > 0) && !c->mat.wall_overlap) {
        ALLOC(c->split, int32_t, n + 1);
        ALLOC(c->mir, int32_t, B + 16);
        ALLOC(c->tb, float, B + 16);
        ALLOC(c->fup, float4, n);
        CK(cudaMemsetAsync(c->dflag, 0, sizeof(unsigned), c->st));
        pair_index(c->rowptr, c->col, n, c->split, c->mir, c->dflag, c->st);
        unsigned bad = 0;
        CK(cudaMemcpyAsync(&bad, c->dflag, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
        s = sync(c);
        if (s) return s;
        if (bad) return fail(c, PD_ECUDA, "bond list is not symmetric");
        c->pairs_ok = true;
        c->pairs = c->opt.pairs == 1;
    }
    CK(cudaGetLastError());
    s = sync(c);
    if (s) return s;
    release(c, k1); release(c, k2); release(c, v1); release(c, v2); release(c, btmp); release(c, cnt);
    c->bonds_ready = true;
    c->list_ok = false;
    // several steps per launch: on request, or by default for problems small enough
    // that one step's launch is mostly fixed cost
    c->persist = c->opt.persistent == 1 || (c->opt.persistent == 0 && n <= PD_PERSIST_AUTO_NODES);
    if (c->opt.lanes_per_node == 0) {
        s = autotune(c);
        if (s) return s;
    } else {
        c->blocks = step_grid(c, c->lanes);
    }
    return eval_forces(c);
}

pd_status pd_set_walls(pd_ctx *c, int nw, const pd_wall *w)
{
    if (!c) return PD_EINVAL;
    if (nw < 0 || nw > PD_MAX_WALLS || (nw > 0 && !w)) return fail(c, PD_EINVAL, "0 <= nw <= 6 walls");
    double pos[PD_MAX_WALLS * 3] = {0}, nrm[PD_MAX_WALLS * 3] = {0};
    WallSet ws;
    memset(&ws, 0, sizeof(ws));
    ws.nw = nw;
    for (int l = 0; l < nw; ++l) {
        double nn = 0;
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(w[l].normal[a]) || !isfinite(w[l].point[a]) || !isfinite(w[l].velocity[a]))
                return fail(c, PD_EINVAL, "non-finite wall data");
            nn += w[l].normal[a] * w[l].normal[a];
        }
        if (fabs(nn - 1.0) > 1e-12) return fail(c, PD_EINVAL, "wall normals must have unit length");
        for (int a = 0; a < 3; ++a) {
            ws.n[l][a] = w[l].normal[a];
            ws.v[l][a] = w[l].velocity[a];
            pos[3 * l + a] = w[l].point[a];
            nrm[3 * l + a] = w[l].normal[a];
        }
    }
    CK(cudaSetDevice(c->opt.device));
    CK(cudaMemcpyAsync(c->wall_pos, pos, sizeof(pos), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->wall_pos + 2 * PD_MAX_WALLS * 3, nrm, sizeof(nrm), cudaMemcpyHostToDevice, c->st));
    CK(reset_impulse(c));
    pd_status s = sync(c);
    if (s) return s;
    c->walls = ws;
    clear_graphs(c);
    if (c->bonds_ready) return eval_forces(c);
    return PD_OK;
}

pd_status pd_get_walls(pd_ctx *c, double *points)
{
    if (!c || (!points && c->walls.nw)) return PD_EINVAL;
    if (!c->walls.nw) return PD_OK;
    CK(cudaMemcpyAsync(points, c->wall_pos, sizeof(double) * 3 * c->walls.nw, cudaMemcpyDeviceToHost, c->st));
    return sync(c);
}

pd_status pd_set_body_force(pd_ctx *c, const double b[3])
{
    if (!c || !b) return PD_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!isfinite(b[a])) return fail(c, PD_EINVAL, "non-finite body force");
    for (int a = 0; a < 3; ++a) c->b[a] = b[a];
    clear_graphs(c);
    if (c->bonds_ready) return eval_forces(c);
    return PD_OK;
}

pd_status pd_stable_dt(pd_ctx *c, double *dt)
{
    if (!c || !dt) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "pd_stable_dt before pd_build_bonds");
    CK(cudaSetDevice(c->opt.device));
    int nb = stable_dt_blocks(c->n);
    stable_dt(c->x4, c->rowptr, c->col, c->n, c->c, c->mat.rho, c->delta, c->mat.micromodulus == 1, c->dscratch,
              c->st);
    std::vector<double> h(nb);
    CK(cudaMemcpyAsync(h.data(), c->dscratch, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
    pd_status s = sync(c);
    if (s) return s;
    double m = INFINITY;
    for (double q : h) m = std::min(m, q);
    *dt = m;
    return PD_OK;
}

// ---- stepping -------------------------------------------------------------------
// Enqueues one chunk of `steps` Verlet steps starting from u[parity]; contact
// lists are rebuilt before the first step and then every k steps.
// Whether pd_step runs its steps between rebuilds in one launch of the multi-step
// kernel: the per-slot global-gather kernels only, not while profiling.
static bool use_persist(const pd_ctx *c)
{
    return c->persist && !c->tiled && !c->pairs && !c->profiling;
}

// Grid of the multi-step kernel: resident blocks, at most one per GPB rows.
static int persist_grid(const pd_ctx *c)
{
    const bool mixed = c->opt.precision == PD_MIXED;
    const bool wx = c->walls.nw > 0 && (c->mat.mu > 0 || (c->mat.wall_overlap && c->walls.nw >= 2));
    const int64_t rows_per_block = 256 / c->lanes;
    const int64_t need = (c->n + rows_per_block - 1) / rows_per_block;
    int b = persist_blocks(c->lanes, c->opt.device, mixed, wx);
    b = (int)std::min<int64_t>({(int64_t)b, (int64_t)c->blocks_cap, need});
    return b;
}

static int64_t enqueue_chunk(pd_ctx *c, int steps, int k, int parity, double dt, bool skip0 = false)
{
    int64_t launches = 0;
    StepParams p = params(c, MODE_FULL, parity, dt);
    launch_drift(p, c->st);
    ++launches;
    int in = parity ^ 1;
    const int pgrid = use_persist(c) ? persist_grid(c) : 0;
    for (int s = 0; s < steps;) {
        if (c->opt.contact && s % k == 0 && !(skip0 && s == 0)) {
            enqueue_rebuild(c, in);
            launches += 12;
        }
        if (pgrid > 0) {
            // the steps up to the next rebuild, all MODE_FULL, in one launch; the
            // chunk's last step (MODE_FINAL) is one k_step launch
            const int run = c->opt.contact ? std::min(k - s % k, steps - s) : steps - s;
            const bool ends = s + run == steps;
            const int full = ends ? run - 1 : run;
            if (full > 1) {
                cudaMemsetAsync(c->gbar, 0, sizeof(unsigned), c->st);
                StepParams pa = params(c, MODE_FULL, in, dt), pb = params(c, MODE_FULL, in ^ 1, dt);
                cudaError_t e =
                    launch_persist(pa, pb, full, c->lanes, pgrid, c->gbar, (unsigned)c->opt.barrier_absent, c->st);
                if (e != cudaSuccess && c->launch_err == cudaSuccess) c->launch_err = e;
                launches += 2;
                if (full & 1) in ^= 1;
            } else if (full == 1) {
                launch_step(params(c, MODE_FULL, in, dt), c->lanes, c->blocks, c->st);
                launches += (c->opt.contact && c->cand_fd) ? 2 : 1;
                in ^= 1;
            }
            s += full;
            if (ends) {
                launch_step(params(c, MODE_FINAL, in, dt), c->lanes, c->blocks, c->st);
                launches += (c->opt.contact && c->cand_fd) ? 2 : 1;
                ++s;
            }
            continue;
        }
        const bool last = (s == steps - 1);
        StepParams q = params(c, last ? MODE_FINAL : MODE_FULL, in, dt);
        const bool prof = c->profiling && c->prof_used + 2 <= (int)c->prof_ev.size();
        if (prof) cudaEventRecord(c->prof_ev[c->prof_used], c->st);
        launch_step(q, c->lanes, c->blocks, c->st);
        if (prof) {
            cudaEventRecord(c->prof_ev[c->prof_used + 1], c->st);
            c->prof_used += 2;
        }
        launches += (c->opt.contact && c->cand_fd) ? 2 : 1;  // the pair-damping kernel runs first
        if (!last) in ^= 1;
        ++s;
    }
    return launches;
}

static pd_status get_graph(pd_ctx *c, int steps, int k, int parity, double dt, bool skip0, GraphEntry **out)
{
    for (auto &g : c->graphs)
        if (g.steps == steps && g.k == k && g.parity == parity && g.skip0 == skip0 && g.dt == dt) {
            *out = &g;
            return PD_OK;
        }
    if (c->graphs.size() >= 6) clear_graphs(c);
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    int64_t launches = enqueue_chunk(c, steps, k, parity, dt, skip0);
    cudaError_t e = cudaStreamEndCapture(c->st, &graph);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(c, PD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e)); }
    GraphEntry ge;
    ge.steps = steps; ge.k = k; ge.parity = parity; ge.skip0 = skip0; ge.dt = dt; ge.launches = launches;
    e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(c, PD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
    c->graphs.push_back(ge);
    *out = &c->graphs.back();
    return PD_OK;
}

#define PD_SEGMENT_CHUNKS 2  // graph chunks per rollback segment of pd_step

static pd_status snapshot(pd_ctx *c, bool restore)
{
    const size_t nb = sizeof(dbl4) * c->n, nf = sizeof(float4) * c->n;
    const bool mixed = c->opt.precision == PD_MIXED;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(restore ? (void *)src : dst, restore ? dst : src, bytes, cudaMemcpyDeviceToDevice, c->st);
    };
    if (mixed) {
        CK(cp(c->snap_rec, c->rec[c->cur], sizeof(float4) * (size_t)rec_float4s(c->n)));
        CK(cp(c->snap_vh, c->vh, nf));
        CK(cp(c->snap_vl, c->vl, nf));
        CK(cp(c->snap_af, c->af, nf));
    } else {
        CK(cp(c->snap_u, c->u[c->cur], nb));
        CK(cp(c->snap_v, c->v, nb));
        CK(cp(c->snap_acc, c->acc, nb));
    }
    CK(cp(c->snap_brk, c->brk, sizeof(uint32_t) * c->nwords));
    CK(cp(c->dscratch + 4096, c->wall_pos, sizeof(double) * PD_MAX_WALLS * 6));
    if (restore) {
        if (c->lcol) sync_lcol_flags(c->brk, c->B, c->lcol, c->st);
        if (c->colf) sync_colf_flags(c->brk, c->col, c->B, c->colf, c->st);
        CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
    }
    return PD_OK;
}

static pd_status rebuild_period(pd_ctx *c, double dt, int *k)
{
    if (!c->opt.contact) { *k = 1 << 30; return PD_OK; }
    // a period the caller fixed is still lowered while a stale list forced it down
    if (c->opt.contact_every > 0) { *k = std::min(c->opt.contact_every, c->k_cap); return PD_OK; }
    int nb = vmax_blocks(c->n);
    if (c->opt.precision == PD_MIXED) materialize_df(c->vh, c->vl, 1, c->n, c->v, c->st);
    vmax(c->v, c->n, c->dscratch, c->st);
    std::vector<double> h(nb);
    CK(cudaMemcpyAsync(h.data(), c->dscratch, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
    pd_status s = sync(c);
    if (s) return s;
    double vm = 0;
    for (double q : h) vm = std::max(vm, q);
    for (int l = 0; l < c->walls.nw; ++l)
        vm = std::max(vm, sqrt(c->walls.v[l][0] * c->walls.v[l][0] + c->walls.v[l][1] * c->walls.v[l][1] +
                               c->walls.v[l][2] * c->walls.v[l][2]));
    // margin on the fastest speed: 1.5x while it is not growing; 2.5x while it
    // grows (a node struck by a moving wall can leave at twice the wall speed)
    const double margin = (c->last_vm > 0 && vm <= 1.05 * c->last_vm) ? 1.5 : 2.5;
    c->last_vm = vm;
    double steps = skin_of(c) / (2.0 * margin * dt * std::max(vm, 1e-30));
    *k = (int)std::max(1.0, std::min({steps, (double)c->opt.graph_chunk, (double)c->k_cap}));
    return PD_OK;
}

// graph chunk length for rebuild period k: the largest multiple of k that fits
// the chunk size, so that rebuilds fall exactly every k steps across chunks
static int chunk_for(const pd_ctx *c, int k)
{
    const int gc = c->opt.graph_chunk;
    return k < gc ? (gc / k) * k : gc;
}

static pd_status run_steps(pd_ctx *c, double dt, int64_t nsteps, int k, int64_t *launches, bool skip0)
{
    int64_t left = nsteps;
    *launches = 0;
    const int chunk = chunk_for(c, k);
    while (left > 0) {
        int steps = (int)std::min<int64_t>(left, chunk);
        const bool sk = skip0 && left == nsteps;  // the first chunk only
        if (use_persist(c)) {  // cooperative launches, enqueued directly (not captured)
            c->launch_err = cudaSuccess;
            *launches += enqueue_chunk(c, steps, std::min(k, steps), c->cur, dt, sk);
            if (c->launch_err != cudaSuccess) {
                cudaGetLastError();
                return fail(c, PD_ECUDA, std::string("multi-step launch: ") + cudaGetErrorString(c->launch_err));
            }
            CK(cudaGetLastError());
            c->cur ^= (steps & 1);
            left -= steps;
            continue;
        }
        if (c->profiling) {
            int kk = std::min(k, steps);
            if ((int)c->prof_ev.size() < c->prof_used + 2 * steps) {
                int want = c->prof_used + 2 * steps;
                while ((int)c->prof_ev.size() < want) {
                    cudaEvent_t e;
                    CK(cudaEventCreate(&e));
                    c->prof_ev.push_back(e);
                }
            }
            *launches += enqueue_chunk(c, steps, kk, c->cur, dt, sk);
            CK(cudaGetLastError());
            c->cur ^= (steps & 1);
            left -= steps;
            continue;
        }
        GraphEntry *g;
        pd_status s = get_graph(c, steps, std::min(k, steps), c->cur, dt, sk, &g);
        if (s) return s;
        CK(cudaGraphLaunch(g->exec, c->st));
        *launches += g->launches;
        c->cur ^= (steps & 1);
        left -= steps;
    }
    return PD_OK;
}

// Steps [t, t + m) as one segment: a rebuild period from the current speeds, a
// snapshot, the graph chunks, one error check.  A segment whose contact list
// went stale or outgrew its capacity is rolled back to its own start and run
// again (shorter rebuild period, larger lists).
static pd_status run_segment(pd_ctx *c, double dt, int64_t left, int64_t *m_out, int64_t *launches, double *ms_out,
                             double *force_ms_out)
{
    // a one-step segment rebuilds at its start whatever the period (no speed
    // readback), unless the list on the device still holds for the current state:
    // then it steps without a rebuild, and the device's stale check decides (a
    // carried list that goes stale sends the step back to be rerun with a rebuild)
    int k = 1;
    pd_status s = left == 1 ? PD_OK : rebuild_period(c, dt, &k);
    if (s) return s;
    bool carry = left == 1 && c->list_ok && c->opt.contact;
    // a rollback costs at most one segment of work
    int64_t m = std::min<int64_t>(left, (int64_t)PD_SEGMENT_CHUNKS * chunk_for(c, k));
    *m_out = m;
    const int cur0 = c->cur;
    s = snapshot(c, false);
    if (s) return s;
    for (int attempt = 0; attempt < 8; ++attempt) {
        c->prof_used = 0;
        CK(cudaEventRecord(c->ev0, c->st));
        s = run_steps(c, dt, m, k, launches, carry);
        if (s) return s;
        CK(cudaEventRecord(c->ev1, c->st));
        if (c->opt.contact) CK(cudaMemcpyAsync(&c->h_stale, c->stale, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        unsigned e = 0;
        s = read_err(c, &e);
        if (s) return s;
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        if (!e) {
            double fm = 0;
            for (int q = 0; q + 1 < c->prof_used; q += 2) {
                float x = 0;
                CK(cudaEventElapsedTime(&x, c->prof_ev[q], c->prof_ev[q + 1]));
                fm += x;
            }
            *ms_out = ms;
            *force_ms_out = fm;
            if (attempt == 0 && c->k_cap < (1 << 29)) c->k_cap *= 2;  // a clean segment relaxes the cap
            c->n_steps += m;
            if (c->opt.contact) {  // each chunk rebuilds at its steps 0, k, 2k, ...
                for (int64_t rest = m; rest > 0; rest -= chunk_for(c, k)) {
                    const int64_t len = std::min<int64_t>(rest, chunk_for(c, k)), kk = std::min<int64_t>(k, len);
                    c->n_rebuilds += (len + kk - 1) / kk;
                }
                if (carry) --c->n_rebuilds;  // ... but the first, with the list carried
            }
            c->list_ok = c->opt.contact && c->h_stale == 0;
            c->t += dt * (double)m;
            c->impulse_span += dt * (double)m;
            return PD_OK;
        }
        c->cur = cur0;
        c->list_ok = false;
        ++c->n_rollbacks;
        s = snapshot(c, true);
        if (s) return s;
        // a stale or overflowed contact list comes first: a node that went through a
        // wall or a non-finite state later in the segment may be its consequence
        if ((e & (PDE_NONFINITE | PDE_WALL | PDE_BARRIER)) && !(e & (PDE_SKIN | PDE_CAPACITY))) {
            c->latched |= e & (PDE_NONFINITE | PDE_WALL | PDE_BARRIER);
            sync(c);
            return status_of(c, e);
        }
        if (e & PDE_CAPACITY) {
            s = grow_candidates(c);
            if (s) return s;
        }
        if (e & PDE_SKIN) {
            if (carry) {  // the carried list went stale: the same step again, from a fresh list
                carry = false;
                continue;
            }
            if (k == 1) return fail(c, PD_ETIMEOUT, "contact list stale even when rebuilt every step");
            k = std::max(1, k / 2);
            c->k_cap = k;  // later segments start from the period that is being tried now
        }
        carry = false;
    }
    return fail(c, PD_ECAPACITY, "pd_step retried too often");
}

pd_status pd_step(pd_ctx *c, double dt, int64_t nsteps)
{
    if (!c) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "pd_step before pd_build_bonds");
    if (c->latched) return fail(c, PD_ESTATE, "a device error is latched; call pd_set_state");
    if (!(dt > 0) || !isfinite(dt) || nsteps < 0) return fail(c, PD_EINVAL, "dt must be > 0 and nsteps >= 0");
    if (c->mat.mu > 0 && c->fric_dt != dt) {
        // the friction's stick branch depends on dt: the acceleration that enters
        // the first half-kick is evaluated again with this dt
        CK(cudaSetDevice(c->opt.device));
        c->fric_dt = dt;
        pd_status s = eval_forces(c);
        if (s) return s;
    }
    if (nsteps == 0) return PD_OK;
    CK(cudaSetDevice(c->opt.device));
    c->last_ms = 0;
    c->last_force_ms = 0;
    c->last_launches = 0;
    for (int64_t done = 0; done < nsteps;) {
        int64_t m = 0, launches = 0;
        double ms = 0, fm = 0;
        pd_status s = run_segment(c, dt, nsteps - done, &m, &launches, &ms, &fm);
        if (s) return s;
        c->last_ms += ms;
        c->last_force_ms += fm;
        c->last_launches += launches;
        done += m;
    }
    return PD_OK;
}


// ---- queries ----------------------------------------------------------------------
pd_status pd_damage(pd_ctx *c, double *phi)
{
    if (!c || !phi) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "pd_damage before pd_build_bonds");
    CK(cudaSetDevice(c->opt.device));
    damage(c->rowptr, c->brk, c->perm, c->n, c->stage, c->st);
    CK(cudaMemcpyAsync(phi, c->stage, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
    return sync(c);
}

// Voigt stress (xx, yy, zz, yz, xz, xy) from wall forces R (nw*3) on areas:
// the wall pushes on the aggregate with -R_l over A_l, whose outward normal is
// m_l = -n_l; sigma e_k = -(R_l / A_l) sign(m_l . e_k) for the dominant axis k
// of m_l, averaged over the walls of each axis, then symmetrised (Sec. 6.4).
static pd_status stress_of(pd_ctx *c, const double *area, const double *R, double sigma[6])
{
    const int nw = c->walls.nw;
    double S[3][3] = {{0}}, cnt[3] = {0, 0, 0};
    for (int l = 0; l < nw; ++l) {
        if (!(area[l] > 0)) return fail(c, PD_EINVAL, "wall areas must be positive");
        double m[3] = {-c->walls.n[l][0], -c->walls.n[l][1], -c->walls.n[l][2]};
        int k = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(m[a]) > fabs(m[k])) k = a;
        const double sg = m[k] > 0 ? 1.0 : -1.0;
        for (int a = 0; a < 3; ++a) S[a][k] += -(R[3 * l + a] / area[l]) * sg;
        cnt[k] += 1;
    }
    for (int k = 0; k < 3; ++k)
        if (cnt[k] > 0)
            for (int a = 0; a < 3; ++a) S[a][k] /= cnt[k];
    double T[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b2 = 0; b2 < 3; ++b2) T[a][b2] = 0.5 * (S[a][b2] + S[b2][a]);
    sigma[0] = T[0][0]; sigma[1] = T[1][1]; sigma[2] = T[2][2];
    sigma[3] = T[1][2]; sigma[4] = T[0][2]; sigma[5] = T[0][1];
    return PD_OK;
}

pd_status pd_bulk_stress(pd_ctx *c, const double *area, double sigma[6], double *wall_force)
{
    if (!c || !sigma) return PD_EINVAL;
    const int nw = c->walls.nw;
    double R[PD_MAX_WALLS * 3] = {0};
    if (nw) {
        if (!area) return fail(c, PD_EINVAL, "area is required when walls are set");
        CK(cudaMemcpyAsync(R, c->react, sizeof(double) * 3 * nw, cudaMemcpyDeviceToHost, c->st));
        pd_status s = sync(c);
        if (s) return s;
    }
    pd_status s = stress_of(c, area, R, sigma);
    if (s) return s;
    if (wall_force)
        for (int q = 0; q < 3 * nw; ++q) wall_force[q] = R[q];
    return PD_OK;
}

pd_status pd_bulk_stress_mean(pd_ctx *c, const double *area, double sigma[6], double *wall_force, double *span)
{
    if (!c || !sigma) return PD_EINVAL;
    const int nw = c->walls.nw;
    double J[PD_MAX_WALLS * 3] = {0}, R[PD_MAX_WALLS * 3] = {0};
    if (nw && !area) return fail(c, PD_EINVAL, "area is required when walls are set");
    const double T = c->impulse_span;
    CK(cudaSetDevice(c->opt.device));
    if (nw) {
        CK(cudaMemcpyAsync(J, c->wall_pos + PD_MAX_WALLS * 3, sizeof(double) * 3 * nw, cudaMemcpyDeviceToHost,
                           c->st));
        CK(reset_impulse(c));
        pd_status s = sync(c);
        if (s) return s;
    }
    c->impulse_span = 0;
    for (int q = 0; q < 3 * nw; ++q) R[q] = T > 0 ? J[q] / T : 0.0;
    pd_status s = stress_of(c, area, R, sigma);
    if (s) return s;
    if (wall_force)
        for (int q = 0; q < 3 * nw; ++q) wall_force[q] = R[q];
    if (span) *span = T;
    return PD_OK;
}

// ---- fragments ------------------------------------------------------------------
// Components of the current state into device scratch (freed by the caller):
// caller-order labels and the fragment index of every label (exclusive scan).
struct FragScratch {
    int32_t *parent = nullptr, *minc = nullptr, *label = nullptr;
    int64_t *is_label = nullptr, *fidx = nullptr;
};

static void frag_release(pd_ctx *c, FragScratch &f)
{
    release(c, f.parent); release(c, f.minc); release(c, f.label); release(c, f.is_label); release(c, f.fidx);
}

static pd_status frag_run(pd_ctx *c, FragScratch &f, int64_t *nfrag)
{
    const int64_t n = c->n;
    ALLOC(f.parent, int32_t, n);
    ALLOC(f.minc, int32_t, n);
    ALLOC(f.label, int32_t, n);
    ALLOC(f.is_label, int64_t, n + 1);
    ALLOC(f.fidx, int64_t, n + 1);
    fragments_device(c->rowptr, c->col, c->brk, c->perm, n, f.parent, f.minc, f.label, f.is_label, c->st);
    scan_exclusive_i64(f.is_label, f.fidx, n, c->tmp, c->st);
    CK(cudaMemcpyAsync(nfrag, f.fidx + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->st));
    return sync(c);
}

pd_status pd_fragments(pd_ctx *c, int32_t *label, int64_t *nfrag)
{
    if (!c || !nfrag) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "pd_fragments before pd_build_bonds");
    CK(cudaSetDevice(c->opt.device));
    FragScratch f;
    pd_status s = frag_run(c, f, nfrag);
    if (!s && label) {
        if (cudaMemcpyAsync(label, f.label, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->st) != cudaSuccess) {
            cudaGetLastError();
            s = fail(c, PD_ECUDA, "fragment label copy failed");
        }
        if (!s) s = sync(c);
    }
    frag_release(c, f);
    return s;
}

pd_status pd_fragment_stats(pd_ctx *c, int64_t nfrag, int64_t *size, double *volume, double *damage)
{
    if (!c || nfrag < 0) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "pd_fragment_stats before pd_build_bonds");
    CK(cudaSetDevice(c->opt.device));
    FragScratch f;
    int64_t have = 0;
    pd_status s = frag_run(c, f, &have);
    if (!s && have != nfrag) s = fail(c, PD_EINVAL, "nfrag does not match the current number of fragments");
    unsigned long long *dsize = nullptr, *dslots = nullptr, *dintact = nullptr;
    double *dvol = nullptr, *ddmg = nullptr;
    FragSortScratch w = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    if (!s && nfrag > 0) {
        const int64_t m = nfrag, n = c->n;
        const int64_t tmpn = std::max(radix_tmp_size(n), scan_tmp_size(m + 1) + 8);
        if (!(dsize = (unsigned long long *)pd_dev_alloc(c, sizeof(unsigned long long) * (m + 1))) ||
            !(dslots = (unsigned long long *)pd_dev_alloc(c, sizeof(unsigned long long) * m)) ||
            !(dintact = (unsigned long long *)pd_dev_alloc(c, sizeof(unsigned long long) * m)) ||
            !(dvol = (double *)pd_dev_alloc(c, sizeof(double) * m)) || !(ddmg = (double *)pd_dev_alloc(c, sizeof(double) * m)) ||
            !(w.k1 = (uint64_t *)pd_dev_alloc(c, sizeof(uint64_t) * n)) ||
            !(w.k2 = (uint64_t *)pd_dev_alloc(c, sizeof(uint64_t) * n)) ||
            !(w.v1 = (uint32_t *)pd_dev_alloc(c, sizeof(uint32_t) * n)) ||
            !(w.v2 = (uint32_t *)pd_dev_alloc(c, sizeof(uint32_t) * n)) ||
            !(w.start = (int64_t *)pd_dev_alloc(c, sizeof(int64_t) * (m + 1))) ||
            !(w.tmp = (int64_t *)pd_dev_alloc(c, sizeof(int64_t) * tmpn))) {
            s = fail(c, PD_ENOMEM, "device allocation failed: fragment statistics");
        } else {
            fragment_stats_device(c->rowptr, c->brk, c->perm, c->x4, f.label, f.fidx, c->n, m, dsize, dvol, dslots,
                                  dintact, ddmg, w, c->st);
            bool ok = true;
            if (size) ok &= cudaMemcpyAsync(size, dsize, sizeof(int64_t) * m, cudaMemcpyDeviceToHost, c->st) == cudaSuccess;
            if (volume) ok &= cudaMemcpyAsync(volume, dvol, sizeof(double) * m, cudaMemcpyDeviceToHost, c->st) == cudaSuccess;
            if (damage) ok &= cudaMemcpyAsync(damage, ddmg, sizeof(double) * m, cudaMemcpyDeviceToHost, c->st) == cudaSuccess;
            if (!ok) { cudaGetLastError(); s = fail(c, PD_ECUDA, "fragment statistics copy failed"); }
            if (!s) s = sync(c);
        }
    }
    release(c, dsize); release(c, dslots); release(c, dintact); release(c, dvol); release(c, ddmg);
    release(c, w.k1); release(c, w.k2); release(c, w.v1); release(c, w.v2); release(c, w.start); release(c, w.tmp);
    frag_release(c, f);
    return s;
}

pd_status pd_num_bonds(pd_ctx *c, int64_t *B)
{
    if (!c || !B) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "no bonds yet");
    *B = c->B;
    return PD_OK;
}

pd_status pd_bonds(pd_ctx *c, int64_t *rowptr, int32_t *col)
{
    if (!c || !rowptr || !col) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "no bonds yet");
    CK(cudaSetDevice(c->opt.device));
    CK(cudaMemcpyAsync(rowptr, c->crow, sizeof(int64_t) * (c->n + 1), cudaMemcpyDeviceToHost, c->st));
    if (c->B) {
        int32_t *tmpc = (int32_t *)pd_dev_alloc(c, sizeof(int32_t) * c->B);
        if (!tmpc) return fail(c, PD_ENOMEM, "pd_bonds staging");
        col_caller(c->col, c->perm, c->kc_of, c->B, tmpc, c->st);
        CK(cudaMemcpyAsync(col, tmpc, sizeof(int32_t) * c->B, cudaMemcpyDeviceToHost, c->st));
        pd_status s = sync(c);
        pd_dev_free(c, tmpc);
        return s;
    }
    return sync(c);
}

pd_status pd_contacts(pd_ctx *c, int64_t *npairs, int32_t *ij)
{
    if (!c || !npairs) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "no bonds yet");
    CK(cudaSetDevice(c->opt.device));
    const int64_t n = c->n;
    for (int attempt = 0; attempt < 4; ++attempt) {
        enqueue_rebuild(c, c->cur);
        unsigned e = 0;
        pd_status s = read_err(c, &e);
        if (s) return s;
        if (e & PDE_CAPACITY) {
            s = grow_candidates(c);
            if (s) return s;
            continue;
        }
        c->list_ok = c->opt.contact != 0;  // rebuilt from the current state
        break;
    }
    int64_t *cnt = (int64_t *)pd_dev_alloc(c, sizeof(int64_t) * (n + 1));
    int64_t *off = (int64_t *)pd_dev_alloc(c, sizeof(int64_t) * (n + 1));
    if (!cnt || !off) { pd_dev_free(c, cnt); pd_dev_free(c, off); return fail(c, PD_ENOMEM, "pd_contacts staging"); }
    const dbl4 *upc = upos(c, c->cur);
    pairs_count(c->x4, upc, c->perm, c->brk, c->cand_ptr, c->cand, n, c->mat.contact_radius, cnt, c->st);
    scan_exclusive_i64(cnt, off, n, c->tmp, c->st);
    int64_t total = 0;
    cudaMemcpyAsync(&total, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->st);
    pd_status s = sync(c);
    if (s == PD_OK && ij) {
        if (total > *npairs) {
            s = fail(c, PD_ECAPACITY, "pair buffer too small");
        } else if (total > 0) {
            int32_t *out = (int32_t *)pd_dev_alloc(c, sizeof(int32_t) * 2 * total);
            if (!out) {
                s = fail(c, PD_ENOMEM, "pd_contacts output");
            } else {
                pairs_fill(c->x4, upc, c->perm, c->brk, c->cand_ptr, c->cand, n, c->mat.contact_radius, off,
                           out, c->st);
                cudaMemcpyAsync(ij, out, sizeof(int32_t) * 2 * total, cudaMemcpyDeviceToHost, c->st);
                s = sync(c);
                pd_dev_free(c, out);
                if (s == PD_OK) {
                    std::vector<std::pair<int32_t, int32_t>> v(total);
                    for (int64_t q = 0; q < total; ++q) v[q] = {ij[2 * q], ij[2 * q + 1]};
                    std::sort(v.begin(), v.end());
                    for (int64_t q = 0; q < total; ++q) { ij[2 * q] = v[q].first; ij[2 * q + 1] = v[q].second; }
                }
            }
        }
    }
    *npairs = total;
    pd_dev_free(c, cnt);
    pd_dev_free(c, off);
    return s;
}

pd_status pd_forces(pd_ctx *c, double *F)
{
    if (!c || !F) return PD_EINVAL;
    if (!c->bonds_ready) return fail(c, PD_ESTATE, "no bonds yet");
    CK(cudaSetDevice(c->opt.device));
    pd_status s = eval_forces(c);
    if (s) return s;
    to_caller(c->F, c->perm, c->n, c->stage, c->st);
    CK(cudaMemcpyAsync(F, c->stage, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, c->st));
    return sync(c);
}

static pd_status get_state_impl(pd_ctx *c, double *u, double *v, uint8_t *broken, uint32_t *bits, double *t)
{
    if (!c) return PD_EINVAL;
    CK(cudaSetDevice(c->opt.device));
    const size_t nb = sizeof(double) * 3 * c->n;
    const bool mixed = c->opt.precision == PD_MIXED;
    if (u) {
        to_caller(upos(c, c->cur), c->perm, c->n, c->stage, c->st);
        CK(cudaMemcpyAsync(u, c->stage, nb, cudaMemcpyDeviceToHost, c->st));
    }
    if (v) {  // a second staging area: no wait for the copy of u
        if (mixed) materialize_df(c->vh, c->vl, 1, c->n, c->v, c->st);
        to_caller(c->v, c->perm, c->n, c->stage + 3 * c->n, c->st);
        CK(cudaMemcpyAsync(v, c->stage + 3 * c->n, nb, cudaMemcpyDeviceToHost, c->st));
    }
    if (broken || bits) {
        if (!c->bonds_ready) return fail(c, PD_ESTATE, "no bonds yet");
        if (c->B && broken) {
            bits_to_bytes(c->brk, c->kc_of, c->B, c->stage_b, c->st);
            CK(cudaMemcpyAsync(broken, c->stage_b, c->B, cudaMemcpyDeviceToHost, c->st));
        } else if (c->B) {  // packed: ceil(B/32) words staged in the byte buffer (B + 16 bytes)
            uint32_t *sw = (uint32_t *)c->stage_b;
            bits_to_packed(c->brk, c->kc_of, c->B, sw, c->st);
            CK(cudaMemcpyAsync(bits, sw, sizeof(uint32_t) * (size_t)((c->B + 31) / 32), cudaMemcpyDeviceToHost,
                               c->st));
        }
    }
    if (t) *t = c->t;
    return sync(c);
}

// Applies a caller state.  Everything given is staged and compared on the device
// with the current state first: non-finite u or v rejects the call; a part that
// applying would leave as it is (on the mixed path the live pairs lie on the FP64
// grid, so what pd_get_state returned, sent back unchanged, splits into exactly
// them) is not applied again, and, for a material without velocity-dependent
// forces, the force evaluation is skipped as well, since the stored acceleration
// is the one an evaluation at this state gives: the run goes on exactly as if the
// call had not been made, which is also how it goes on from the applied state.
// With damping or friction the stored acceleration saw the half-step velocity of
// the last step, so it is evaluated again.
static pd_status set_state_impl(pd_ctx *c, const double *u, const double *v, const uint8_t *broken,
                                const uint32_t *bits, const double *t)
{
    if (!c) return PD_EINVAL;
    CK(cudaSetDevice(c->opt.device));
    if ((broken || bits) && !c->bonds_ready) return fail(c, PD_ESTATE, "no bonds yet");
    const size_t nb = sizeof(double) * 3 * c->n;
    const bool mixed = c->opt.precision == PD_MIXED;
    const bool with_bits = (broken || bits) && c->B > 0;
    double *su = c->stage, *sv = c->stage + 3 * c->n;
    unsigned flags = 0;
    if (u || v || with_bits) {
        CK(cudaMemsetAsync(c->dflag, 0, sizeof(unsigned), c->st));
        if (u) {
            CK(cudaMemcpyAsync(su, u, nb, cudaMemcpyHostToDevice, c->st));
            check_finite(su, 3 * c->n, 1u, c->dflag, c->st);
            state_differs(su, c->perm, c->n, mixed ? c->uh[c->cur] : nullptr, mixed ? c->ul[c->cur] : nullptr, REC,
                          c->u[c->cur], 4u, c->dflag, c->st);
        }
        if (v) {
            CK(cudaMemcpyAsync(sv, v, nb, cudaMemcpyHostToDevice, c->st));
            check_finite(sv, 3 * c->n, 2u, c->dflag, c->st);
            state_differs(sv, c->perm, c->n, mixed ? c->vh : nullptr, mixed ? c->vl : nullptr, 1, c->v, 8u, c->dflag,
                          c->st);
        }
        if (with_bits) {
            const int64_t nw = (c->B + 31) / 32;
            if (broken) {  // the caller's bytes in internal slot order, compared with the live bits
                CK(cudaMemcpyAsync(c->stage_b, broken, c->B, cudaMemcpyHostToDevice, c->st));
                bytes_to_bits(c->stage_b, c->kc_of, c->B, c->stage_bits, c->st);
                words_differ(c->stage_bits, c->brk, nw, 0xffffffffu, 16u, c->dflag, c->st);
            } else {  // the live bits in caller order (cheap: breaks are sparse), compared with the caller's
                uint32_t *sw = (uint32_t *)c->stage_b;
                CK(cudaMemcpyAsync(sw, bits, sizeof(uint32_t) * (size_t)nw, cudaMemcpyHostToDevice, c->st));
                bits_to_packed(c->brk, c->kc_of, c->B, c->stage_bits, c->st);
                const uint32_t last = (c->B & 31) ? (1u << (c->B & 31)) - 1u : 0xffffffffu;  // bits past B ignored
                words_differ(sw, c->stage_bits, nw, last, 16u, c->dflag, c->st);
            }
        }
        CK(cudaMemcpyAsync(&flags, c->dflag, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
        pd_status s = sync(c);
        if (s) return s;
        if (flags & 1u) return fail(c, PD_EINVAL, "u contains a non-finite value");
        if (flags & 2u) return fail(c, PD_EINVAL, "v contains a non-finite value");
    }
    const bool changed = (flags & (4u | 8u | 16u)) != 0;
    if (u && (flags & 4u)) {
        if (mixed) {
            from_caller(su, c->perm, c->n, c->u[0], c->st);
            split_df(c->u[0], c->xl4, c->n, c->uh[c->cur], c->ul[c->cur], REC, c->st);
        } else {
            from_caller(su, c->perm, c->n, c->u[c->cur], c->st);
        }
    }
    if (v && (flags & 8u)) {
        from_caller(sv, c->perm, c->n, c->v, c->st);
        if (mixed) split_df(c->v, nullptr, c->n, c->vh, c->vl, 1, c->st);
    }
    if (with_bits && (flags & 16u)) {
        if (bits) packed_to_bits((const uint32_t *)c->stage_b, c->kc_of, c->B, c->stage_bits, c->st);
        CK(cudaMemcpyAsync(c->brk, c->stage_bits, sizeof(uint32_t) * (size_t)((c->B + 31) / 32),
                           cudaMemcpyDeviceToDevice, c->st));
        if (c->lcol) sync_lcol_flags(c->brk, c->B, c->lcol, c->st);
        if (c->colf) sync_colf_flags(c->brk, c->col, c->B, c->colf, c->st);
    }
    if (t) c->t = *t;
    c->latched = 0;
    CK(cudaMemsetAsync(c->derr, 0, sizeof(unsigned), c->st));
    CK(reset_impulse(c));  // stream-ordered before any later work; the evaluation below synchronises
    const bool velocity_forces = c->mat.beta_d > 0 || c->mat.mu > 0;
    const bool skip = !changed && !velocity_forces;
    ++(skip ? c->n_state_unchanged : c->n_state_applied);
    if (c->bonds_ready && !skip) return eval_forces(c);
    return PD_OK;
}

pd_status pd_get_state(pd_ctx *c, double *u, double *v, uint8_t *broken, double *t)
{
    return get_state_impl(c, u, v, broken, nullptr, t);
}

pd_status pd_set_state(pd_ctx *c, const double *u, const double *v, const uint8_t *broken, const double *t)
{
    return set_state_impl(c, u, v, broken, nullptr, t);
}

pd_status pd_get_state_packed(pd_ctx *c, double *u, double *v, uint32_t *broken_bits, double *t)
{
    return get_state_impl(c, u, v, nullptr, broken_bits, t);
}

pd_status pd_set_state_packed(pd_ctx *c, const double *u, const double *v, const uint32_t *broken_bits,
                              const double *t)
{
    return set_state_impl(c, u, v, nullptr, broken_bits, t);
}

pd_status pd_tuning(pd_ctx *c, int *lanes, int *kernel, double ms[12])
{
    if (!c) return PD_EINVAL;
    if (lanes) *lanes = c->lanes;
    if (kernel) *kernel = c->pairs ? 2 : (c->tiled ? 1 : 0);
    if (ms)
        for (int q = 0; q < 12; ++q) ms[q] = c->tune_ms[q];
    return PD_OK;
}

pd_status pd_set_profiling(pd_ctx *c, int on)
{
    if (!c) return PD_EINVAL;
    c->profiling = on != 0;
    return PD_OK;
}

pd_status pd_step_counters(pd_ctx *c, int64_t *steps, int64_t *rebuilds, int64_t *rollbacks)
{
    if (!c) return PD_EINVAL;
    if (steps) *steps = c->n_steps;
    if (rebuilds) *rebuilds = c->n_rebuilds;
    if (rollbacks) *rollbacks = c->n_rollbacks;
    return PD_OK;
}

pd_status pd_state_counters(pd_ctx *c, int64_t *applied, int64_t *unchanged)
{
    if (!c) return PD_EINVAL;
    if (applied) *applied = c->n_state_applied;
    if (unchanged) *unchanged = c->n_state_unchanged;
    return PD_OK;
}

pd_status pd_last_step_stats(pd_ctx *c, double *ms_force, double *ms_total, int64_t *launches)
{
    if (!c) return PD_EINVAL;
    if (ms_force) *ms_force = c->last_force_ms;
    if (ms_total) *ms_total = c->last_ms;
    if (launches) *launches = c->last_launches;
    return PD_OK;
}

}  // extern "C"
