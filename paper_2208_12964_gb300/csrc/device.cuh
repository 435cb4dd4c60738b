// Device building blocks of the per-view MART kernels, shared by the
// single-reconstruction kernels (mart.cu) and the batched kernels (batch.cu).
#pragma once

#include "internal.cuh"

namespace uspg {

// ---- programmatic dependent launch -------------------------------------------
//
// The per-view kernels are launched so that each may start while the one
// before it on the stream drains (programmatic stream serialization).  Each
// reads only static data (store, tables) before this wait, and everything
// the previous kernel wrote after it; without such a launch the wait returns
// at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ---- weight loads ------------------------------------------------------------

__device__ __forceinline__ float load_w1(const float *w, long long q) { return w[q]; }
__device__ __forceinline__ float load_w1(const __half *w, long long q) { return __half2float(w[q]); }
__device__ __forceinline__ float load_w1(const __nv_bfloat16 *w, long long q) { return __bfloat162float(w[q]); }

// rotated cell id of a stored entry; tab[ring] = {head, ng, q, 0}
__device__ __forceinline__ long long rot_cell(const int4 *tab, long long cps, uint32_t pc)
{
    int4 t = tab[cell_ring(pc)];
    int s = cell_sector(pc) + t.z;
    s = s >= t.y ? s - t.y : s;
    return (long long)cell_slab(pc) * cps + t.x + s;
}

// rotated position of a stored entry within its slab (head + sector)
__device__ __forceinline__ int rot_within(const int4 *tab, uint32_t pc)
{
    int4 t = tab[cell_ring(pc)];
    int s = cell_sector(pc) + t.z;
    s = s >= t.y ? s - t.y : s;
    return t.x + s;
}

__device__ __forceinline__ void fill_tab(int4 *tab, const RingEntry *rt, int n_rings, int mG, int tid, int nt)
{
    for (int i = tid; i < n_rings; i += nt) {
        RingEntry e = rt[i];
        tab[i] = make_int4(e.head, e.ng, mG * e.step, 0);
    }
}

__device__ __forceinline__ void load_w8(const float *w, long long q, float o[8])
{
    float4 a = __ldcs((const float4 *)(w + q)), b = __ldcs((const float4 *)(w + q + 4));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void load_w8(const __half *w, long long q, float o[8])
{
    uint4 u = __ldcs((const uint4 *)(w + q));
    const __half2 *h = (const __half2 *)&u;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 v = __half22float2(h[i]);
        o[2 * i] = v.x;
        o[2 * i + 1] = v.y;
    }
}
__device__ __forceinline__ void load_w8(const __nv_bfloat16 *w, long long q, float o[8])
{
    uint4 u = __ldcs((const uint4 *)(w + q));
    const __nv_bfloat162 *h = (const __nv_bfloat162 *)&u;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float2 v = __bfloat1622float2(h[i]);
        o[2 * i] = v.x;
        o[2 * i + 1] = v.y;
    }
}
__device__ __forceinline__ float load_cs(const float *w, long long q) { return __ldcs(w + q); }
__device__ __forceinline__ float load_cs(const __half *w, long long q)
{
    return __half2float(__ushort_as_half(__ldcs((const unsigned short *)(w + q))));
}
__device__ __forceinline__ float load_cs(const __nv_bfloat16 *w, long long q)
{
    return __bfloat162float(__ushort_as_bfloat16(__ldcs((const unsigned short *)(w + q))));
}

template <typename WT>
struct Group8 {
    uint32_t c[8];
    float w[8];
    uint32_t ray;
};

template <typename WT>
__device__ __forceinline__ void load_group(Group8<WT> &G, const uint32_t *idx, const WT *w, const uint32_t *grp_ray,
                                           long long g, bool valid)
{
    if (valid) {
        long long q = g * kRowPad;
        uint4 ia = __ldcs((const uint4 *)(idx + q)), ib = __ldcs((const uint4 *)(idx + q + 4));
        load_w8(w, q, G.w);
        G.ray = __ldcs(grp_ray + g);
        G.c[0] = ia.x; G.c[1] = ia.y; G.c[2] = ia.z; G.c[3] = ia.w;
        G.c[4] = ib.x; G.c[5] = ib.y; G.c[6] = ib.z; G.c[7] = ib.w;
    } else {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            G.c[i] = 0;
            G.w[i] = 0.0f;
        }
        G.ray = 0xffffffffu;
    }
}

// Forward ray sums over the 8-entry groups [0, n_groups) of one
// representative's rows (group g starts at entry (g0 + g) * 8), by warps
// w = wg, wg + W, ...; partial sums of each ray segment go to sacc[ray].
// tab: ring table {head, ng, shift} of the view.  Each lane takes one group;
// the next chunk's stream loads are issued before the current chunk's image
// gathers, and lanes of the same ray are combined by a segmented shuffle sum.
// MIR (z-mirror store): every stored row also yields the sum of its mirror
// ray, from the same entries with the slab flipped; a row that is its own
// mirror adds once.  PAIRS: the image is in the mirrored pair layout, so one
// 8-byte gather gives a cell and its mirror.
template <typename WT, bool MIR, bool PAIRS = MIR>
__device__ __forceinline__ void fwd_groups(const uint32_t *__restrict__ idx, const WT *__restrict__ w,
                                           const uint32_t *__restrict__ grp_ray, long long g0, long long n_groups,
                                           const float *__restrict__ f, const int4 *tab, long long cps,
                                           float *__restrict__ sacc, long long wg, long long W, int lane,
                                           const Mirror &M)
{
    const long long step = W * 32;
    long long base = wg * 32;
    if (base >= n_groups) return;
    Group8<WT> cur, nxt;
    load_group(cur, idx, w, grp_ray, g0 + base + lane, base + lane < n_groups);
    grid_dep_wait();  // the image and the accumulator belong to the previous kernels
    for (; base < n_groups; base += step) {
        long long nb = base + step;
        load_group(nxt, idx, w, grp_ray, g0 + nb + lane, nb + lane < n_groups);
        float acc = 0.0f, accm = 0.0f;
        if (MIR && PAIRS) {
            float2 gp[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                int sl = cell_slab(cur.c[i]);
                int lo = 2 * sl <= M.n_slabs - 1 ? sl : M.n_slabs - 1 - sl;  // pair row: the lower slab
                long long k = (long long)lo * cps + rot_within(tab, cur.c[i]);
                gp[i] = cur.w[i] != 0.0f ? __ldg((const float2 *)f + k) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int i = 0; i < 8; i++) {
                bool low = 2 * cell_slab(cur.c[i]) <= M.n_slabs - 1;
                acc = fmaf(cur.w[i], low ? gp[i].x : gp[i].y, acc);
                accm = fmaf(cur.w[i], low ? gp[i].y : gp[i].x, accm);
            }
        } else if (MIR) {
            float gv[8], gm[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                bool on = cur.w[i] != 0.0f;
                long long cl = rot_cell(tab, cps, cur.c[i]);
                long long cm = cl + (long long)(M.n_slabs - 1 - 2 * cell_slab(cur.c[i])) * cps;
                gv[i] = on ? __ldg(f + cl) : 0.0f;
                gm[i] = on ? __ldg(f + cm) : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 8; i++) {
                acc = fmaf(cur.w[i], gv[i], acc);
                accm = fmaf(cur.w[i], gm[i], accm);
            }
        } else {
            float gv[8];
#pragma unroll
            for (int i = 0; i < 8; i++) gv[i] = cur.w[i] != 0.0f ? __ldg(f + rot_cell(tab, cps, cur.c[i])) : 0.0f;
#pragma unroll
            for (int i = 0; i < 8; i++) acc = fmaf(cur.w[i], gv[i], acc);
        }
        uint32_t ray = cur.ray;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            float v2 = __shfl_down_sync(0xffffffffu, acc, o);
            float m2 = MIR ? __shfl_down_sync(0xffffffffu, accm, o) : 0.0f;
            uint32_t r2 = __shfl_down_sync(0xffffffffu, ray, o);
            if (lane + o < 32 && r2 == ray) {
                acc += v2;
                accm += m2;
            }
        }
        uint32_t rprev = __shfl_up_sync(0xffffffffu, ray, 1);
        if (ray != 0xffffffffu && (lane == 0 || rprev != ray)) {
            atomicAdd(&sacc[ray], acc);
            if (MIR) {
                int rm = mirror_ray((int)ray, M.n_u, M.n_v);
                if (rm != (int)ray) atomicAdd(&sacc[rm], accm);
            }
        }
        cur = nxt;
    }
}

// Per-view update rule of the correction kernels (Sec. III.D):
//  power (linear == 0): f *= exp(lambda * sum w ln(P/Pbar) / sum w), the
//      weighted geometric mean of the view's ray ratios;
//  Eq. 18 (linear == 1): f *= sum w (1 - lambda (1 - P/Pbar)) / sum w, the
//      weighted arithmetic mean of the rays' Eq. 18 factors.
// tol > 0 (Eq. 19): every cell whose correction moves it by more than
// tol * |f_old| sets *moved.
struct UpdateRule {
    float lambda;
    int linear;
    float tol;
    int *moved;
};

// The ray value the correction averages: ln(P/Pbar) (power rule; -inf for
// P = 0, which zeroes the cells of the ray) or P/Pbar (Eq. 18).  NaN marks a
// ray to skip: empty row or zero sum, or a projection that is not a finite
// non-negative number (such data are refused at input; a ray that carries
// one anyway changes nothing).
__device__ __forceinline__ float ray_value(float sv, float p, int linear)
{
    if (!(sv > 0.0f) || !(p >= 0.0f && p <= 3.402823466e38f)) return __int_as_float(0x7fc00000);
    if (linear) return p / sv;
    return p > 0.0f ? logf(p / sv) : -INFINITY;
}

// What the correction adds per unit weight for one ray: (value, 1) for a ray
// that takes part, (0, 0) for a skipped one, so that a cell's sums are plain
// fused multiply-adds, num += w * x and den += w * y.  A ray with P = 0
// (power rule) carries -inf and makes num -inf: the cell becomes 0.
__device__ __forceinline__ float2 ray_term(float sv, float p, int linear)
{
    float r = ray_value(sv, p, linear);
    return r == r ? make_float2(r, 1.0f) : make_float2(0.0f, 0.0f);
}

// Ray term of one ray from its accumulated sum; clears the accumulator.
__device__ __forceinline__ void finalize_ray(float *__restrict__ sacc, const float *__restrict__ proj, int ray,
                                             float w_scale, int linear, float *__restrict__ out_s,
                                             float2 *__restrict__ out_res)
{
    float sv = sacc[ray] * w_scale;
    sacc[ray] = 0.0f;
    if (out_s) out_s[ray] = sv;
    if (out_res) out_res[ray] = ray_term(sv, proj[ray], linear);
}

// z-mirror store: stored ray r and its mirror m.  The terms are written in
// both orders, out_res4[r] = {term of r, term of m} and
// out_res4[r + n_rows] = {term of m, term of r}: a column entry's key is the
// index of the pair whose first half its own cell sees (and whose second half
// the cell's mirror sees), so one 16-byte gather serves both cells.
__device__ __forceinline__ void finalize_pair(float *__restrict__ sacc, const float *__restrict__ proj, int ray,
                                              const Mirror &M, float w_scale, int linear, float *__restrict__ out_s,
                                              float4 *__restrict__ out_res4)
{
    int rm = mirror_ray(ray, M.n_u, M.n_v);
    float sv = sacc[ray] * w_scale;
    float sm = rm != ray ? sacc[rm] * w_scale : sv;
    sacc[ray] = 0.0f;
    sacc[rm] = 0.0f;
    if (out_s) {
        out_s[ray] = sv;
        out_s[rm] = sm;
    }
    if (out_res4) {
        float2 t = ray_term(sv, proj[ray], linear), tm = ray_term(sm, proj[rm], linear);
        out_res4[ray] = make_float4(t.x, t.y, tm.x, tm.y);
        out_res4[ray + M.n_rows] = make_float4(tm.x, tm.y, t.x, t.y);
    }
}

// New value of a cell met by at least one ray (den > 0).  Power rule:
// f * exp(lambda * num / den), 0 if one of its rays has P = 0; Eq. 18:
// f * (1 - lambda + lambda * num / den).  The ratio is a weighted mean, so
// the fast reciprocal and exponential (a few units in the last place) are far
// inside the image tolerance.
__device__ __forceinline__ float cell_update(float fv, float num, float den, bool zero, const UpdateRule &U)
{
    float m = __fdividef(num, den);
    if (U.linear) return fv * fmaf(U.lambda, m, 1.0f - U.lambda);
    return zero ? 0.0f : fv * __expf(U.lambda * m);
}

// Eq. 19: does the correction fv -> nv break |nv - fv| <= tol |fv|?
__device__ __forceinline__ bool moved_cell(float fv, float nv, const UpdateRule &U)
{
    return U.tol > 0.0f && fabsf(nv - fv) > U.tol * fabsf(fv);
}

// Per-lane correction sums of one cell (and, MIR, of its mirror cell).
struct CellSums {
    float num, den, numm, denm;
};

// Adds one column entry of weight w: term = {x, y} of the ray the cell sees
// (and, MIR, {z, w} of the ray its mirror sees).  Absent rows have w = 0 and
// a zero term; a stored entry has w > 0 (weights that round to 0 in a
// reduced-precision store are left out of the cell-major store), so an
// infinite term never meets a zero weight.
__device__ __forceinline__ void add_term(float w, float4 t, CellSums &S)
{
    S.num = fmaf(w, t.x, S.num);
    S.den = fmaf(w, t.y, S.den);
    S.numm = fmaf(w, t.z, S.numm);
    S.denm = fmaf(w, t.w, S.denm);
}
__device__ __forceinline__ void add_term(float w, float2 t, CellSums &S)
{
    S.num = fmaf(w, t.x, S.num);
    S.den = fmaf(w, t.y, S.den);
}

// Rows 0..R-1 of one lane (kp, wp: the lane's entry in row 0; row t is
// t * 32 entries on): loads first, then the ray-term gathers, then the sums.
// MIR: the key indexes the pair table written by finalize_pair; otherwise
// the key is the ray and the table holds one term per ray.
template <typename WT, bool MIR, int R>
__device__ __forceinline__ void cm_rows(const uint32_t *kp, const WT *wp, const float *res, int cnt, CellSums &S)
{
    uint32_t ky[R];
    float wv[R];
#pragma unroll
    for (int t = 0; t < R; t++) {
        bool in = t < cnt;
        ky[t] = in ? __ldcs(kp + t * kSlice) : 0u;
        wv[t] = in ? load_cs(wp, t * kSlice) : 0.0f;
    }
    if (MIR) {
        float4 rv[R];
#pragma unroll
        for (int t = 0; t < R; t++) rv[t] = t < cnt ? __ldg((const float4 *)res + ky[t]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < R; t++) add_term(wv[t], rv[t], S);
    } else {
        float2 rv[R];
#pragma unroll
        for (int t = 0; t < R; t++) rv[t] = t < cnt ? __ldg((const float2 *)res + ky[t]) : make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < R; t++) add_term(wv[t], rv[t], S);
    }
}

// The correction is latency-bound (about 1.6 entries per cell and view, at
// most a few per slice row): 8 resident blocks of 256 threads (32 registers
// a thread, 64 warps per SM) hide more of it than fewer, fatter warps; rows
// are unrolled by 2 or 4 (a loop beyond) to stay within those registers.
constexpr int kBwdMinBlocks = 8;
constexpr int kBwdMinBlocksMirror = 6;  // the mirrored form holds two cells per lane

// Correction of slices wg, wg + W, ... of one representative (lane-ordered
// cell-major store): each lane owns one cell; the next slice's descriptors
// are loaded before the current slice's stream; the unrolled row loop is
// sized per slice from lane 0's (widest) count.  sdesc[s] = {first slot of
// slice s relative to cray / cw, meta}; lane_desc[32 s + l] = (source lane
// << 11) | count; tab: ring table {head, ng, shift, 0} of the view.  MIR: the
// store holds the lower-half and middle slabs; a lane also updates the mirror
// cell (slab n_s-1-s) from the same column, except in the middle slab.  All
// index arithmetic is 32-bit (slices * 32 and cell ids are below 2^31).
template <typename WT, bool MIR>
__device__ __forceinline__ void bwd_slices(const uint2 *__restrict__ sdesc, const uint16_t *__restrict__ lane_desc,
                                           const uint32_t *__restrict__ cray, const WT *__restrict__ cw,
                                           const float *__restrict__ res, float *__restrict__ f, const int4 *tab,
                                           uint32_t cps, int n_slices, const UpdateRule &U, int wg, int W, int lane,
                                           const Mirror &M)
{
    int sl = wg;
    if (sl >= n_slices) return;
    uint2 dn = sdesc[sl];
    uint32_t ln = lane_desc[sl * kSlice + lane];
    grid_dep_wait();  // the ray terms and the image belong to the previous kernels
    for (; sl < n_slices; sl += W) {
        const uint2 dc = dn;
        const uint32_t lc = ln;
        if (sl + W < n_slices) {
            dn = sdesc[sl + W];
            ln = lane_desc[(sl + W) * kSlice + lane];
        }
        const int cnt = (int)(lc & 2047u);
        const int width = __shfl_sync(0xffffffffu, cnt, 0);
        const int4 t = tab[cell_ring(dc.y)];
        int sec = cell_sector(dc.y) + (int)(lc >> 11) + t.z;
        sec = sec >= t.y ? sec - t.y : sec;
        const int slab = cell_slab(dc.y);
        const uint32_t k = (uint32_t)slab * cps + (uint32_t)(t.x + sec);  // MIR: the pair {cell, mirror cell}
        const bool pair = MIR && 2 * slab != M.n_slabs - 1;                // the middle slab is its own mirror
        float fv = 0.0f, fm = 0.0f;
        if (cnt > 0) {
            if (MIR) {
                float2 v = ((const float2 *)f)[k];
                fv = v.x;
                fm = v.y;
            } else {
                fv = f[k];
            }
        }
        const uint32_t *kp = cray + (dc.x + lane);
        const WT *wp = cw + (dc.x + lane);
        CellSums S{0.f, 0.f, 0.f, 0.f};
        if (width <= 2) {
            cm_rows<WT, MIR, 2>(kp, wp, res, cnt, S);
        } else {
            cm_rows<WT, MIR, 4>(kp, wp, res, cnt, S);
            for (int r = 4; r < cnt; r++) {  // long columns (cells close to the source)
                float wt = load_cs(wp, r * kSlice);
                uint32_t key = __ldcs(kp + r * kSlice);
                if (MIR) add_term(wt, __ldg((const float4 *)res + key), S);
                else add_term(wt, __ldg((const float2 *)res + key), S);
            }
        }
        // a ray with P = 0 has made num -inf (power rule): the cell becomes 0
        float nx = S.den > 0.0f ? cell_update(fv, S.num, S.den, S.num == -INFINITY, U) : fv;
        float ny = fm;
        if (MIR) {
            ny = !pair ? nx : (S.denm > 0.0f ? cell_update(fm, S.numm, S.denm, S.numm == -INFINITY, U) : fm);
            if (S.den > 0.0f || (pair && S.denm > 0.0f)) ((float2 *)f)[k] = make_float2(nx, ny);
        } else if (S.den > 0.0f) {
            f[k] = nx;
        }
        if (U.tol > 0.0f) {  // Eq. 19 (uniform branch)
            bool mv = moved_cell(fv, nx, U) || (MIR && moved_cell(fm, ny, U));
            if (__any_sync(0xffffffffu, mv) && lane == 0) *U.moved = 1;
        }
    }
}

}  // namespace uspg
