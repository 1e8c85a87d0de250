// Host launchers of the set-up and rebuild kernels (pd_build.cu).
#pragma once

#include "pd_grid.cuh"
#include "pd_internal.cuh"

#define PD_MAX_FILTERS 8

struct FilterSet {
    int nf;
    int kind[PD_MAX_FILTERS];
    double a[PD_MAX_FILTERS][12];
};

void build_morton(const double *x_dev, int64_t n, const double lo[3], const double hi[3], uint64_t *key,
                  uint64_t *key_alt, uint32_t *val, uint32_t *val_alt, int grain_bits, const int32_t *grain_dev,
                  int64_t *tmp, uint32_t **order_out, cudaStream_t st);
void gather_nodes(const uint32_t *order, int64_t n, const double *x, const double *vol, const int32_t *grain,
                  const double *v0, int32_t *perm, int32_t *inv, dbl4 *x4, int32_t *grain_out, dbl4 *v,
                  float4 *xh4, float4 *xl4, const double centre[3], cudaStream_t st);
void bonds_count(const dbl4 *x4, const int32_t *grain, const int32_t *perm, int64_t n, const GridView &g,
                 double delta, const FilterSet &f, int64_t *cnt, cudaStream_t st);
void bonds_fill(const dbl4 *x4, const int32_t *grain, const int32_t *perm, int64_t n, const GridView &g,
                double delta, const FilterSet &f, const int64_t *off, uint64_t *keys, int sh, cudaStream_t st);
void bonds_keys_to_col(const uint64_t *keys, int64_t B, int sh, int32_t *col, cudaStream_t st);
void cand_count(const dbl4 *x4, const dbl4 *u4, const int32_t *grain, const int64_t *rowptr, const int32_t *col,
                int64_t n, const GridView &g, double cut, int64_t *cnt, cudaStream_t st);
void cand_fill(const dbl4 *x4, const dbl4 *u4, const int32_t *grain, const int64_t *rowptr, const int32_t *col,
               int64_t n, const GridView &g, double cut, const int64_t *off, int2 *cand, int64_t cap, unsigned *err,
               double *disp, int *stale, cudaStream_t st);
void pairs_count(const dbl4 *x4, const dbl4 *u4, const int32_t *perm, const uint32_t *brk, const int64_t *cp,
                 const int2 *cand, int64_t n, double Rc, int64_t *cnt, cudaStream_t st);
void pairs_fill(const dbl4 *x4, const dbl4 *u4, const int32_t *perm, const uint32_t *brk, const int64_t *cp,
                const int2 *cand, int64_t n, double Rc, const int64_t *off, int32_t *out, cudaStream_t st);
void damage(const int64_t *rowptr, const uint32_t *brk, const int32_t *perm, int64_t n, double *phi,
            cudaStream_t st);
int stable_dt_blocks(int64_t n);
void stable_dt(const dbl4 *x4, const int64_t *rowptr, const int32_t *col, int64_t n, double c, double rho,
               double delta, int conic, double *partial, cudaStream_t st);
void canon_keys(const int64_t *rowptr, const int32_t *col, const int32_t *perm, int64_t n, int sh, uint64_t *keys,
                uint32_t *vals, cudaStream_t st);
void canon_invert(const uint32_t *vals, int64_t B, int32_t *kc_of, cudaStream_t st);
void row_len_caller(const int64_t *rowptr, const int32_t *inv, int64_t n, int64_t *len, cudaStream_t st);
void col_caller(const int32_t *col, const int32_t *perm, const int32_t *kc_of, int64_t B, int32_t *out,
                cudaStream_t st);
void bits_to_bytes(const uint32_t *brk, const int32_t *kc_of, int64_t B, uint8_t *out, cudaStream_t st);
void bytes_to_bits(const uint8_t *in, const int32_t *kc_of, int64_t B, uint32_t *brk, cudaStream_t st);
// the same in packed form: bit c % 32 of word c / 32 for canonical slot c (ceil(B/32) words)
void bits_to_packed(const uint32_t *brk, const int32_t *kc_of, int64_t B, uint32_t *out, cudaStream_t st);
void packed_to_bits(const uint32_t *in, const int32_t *kc_of, int64_t B, uint32_t *brk, cudaStream_t st);
void to_caller(const dbl4 *in, const int32_t *perm, int64_t n, double *out, cudaStream_t st);
void from_caller(const double *in, const int32_t *perm, int64_t n, dbl4 *out, cudaStream_t st);
// *flag |= bit when the caller-order state `staged` (n*3) differs from the current
// one: double-float pairs hi/lo (stride in float4) when hi != NULL, else d64
void state_differs(const double *staged, const int32_t *perm, int64_t n, const float4 *hi, const float4 *lo,
                   int stride, const dbl4 *d64, unsigned bit, unsigned *flag, cudaStream_t st);
// *flag |= bit when the nw words of a and b differ
// flag |= bit when the words differ (the last word only in the bits of last_mask)
void words_differ(const uint32_t *a, const uint32_t *b, int64_t nw, uint32_t last_mask, unsigned bit, unsigned *flag,
                  cudaStream_t st);
// *flag |= bit when any of the m doubles at a is not finite
void check_finite(const double *a, int64_t m, unsigned bit, unsigned *flag, cudaStream_t st);
void split_hilo(const dbl4 *u, int64_t n, float4 *hi, float4 *lo, cudaStream_t st);
int vmax_blocks(int64_t n);
void vmax(const dbl4 *v, int64_t n, double *partial, cudaStream_t st);
// Shared-memory tiles of T consecutive rows: sorted unique node list per tile
// (ulist, tile_ptr[ntiles+1]) and tile-local indices of bond targets (lcol) and
// rows (lrow); 0xffff marks tiles whose list exceeds cap.  ulist must hold B + n.
void build_tiles(const int64_t *rowptr, const int32_t *col, int64_t n, int64_t B, int T, int sh, int cap,
                 uint64_t *keys, uint64_t *keys_alt, int64_t *flag, int64_t *pos, int64_t *tmp, int32_t *ulist,
                 int64_t *tile_ptr, uint16_t *lcol, uint16_t *lrow, cudaStream_t st);
void sync_lcol_flags(const uint32_t *brk, int64_t B, uint16_t *lcol, cudaStream_t st);
void sync_colf_flags(const uint32_t *brk, const int32_t *col, int64_t B, int32_t *colf, cudaStream_t st);
// split (n) and mirror slots (B) of the each-bond-once passes; *bad |= 1 if a bond lacks its reverse
void pair_index(const int64_t *rowptr, const int32_t *col, int64_t n, int32_t *split, int32_t *mir, unsigned *bad,
                cudaStream_t st);
