// Grouped full single links, mixed form (the links kernel and the full part
// of the batched kernel).  See links_full.cu for the formulas.
#pragma once

#include "links_tile.cuh"

namespace lisa {

// ---------------------------------------------------------------------------
// Mixed form, grouped: one CTA per group of up to 8 tiles (as many as keep the
// group's half-span within 1.1e4 s, the LFA kernel's bound for in-group
// cubics) around one FP64 set-up at the group centre: the twelve link-time
// splits and their FP32 cubics, and n_l - k with its cubics.  The group runs
// in sub-blocks of two tiles, each thread computing samples t and kTile + t of
// the sub-block; the two samples' Lagrange weights are formed together in
// packed FP32 pair instructions (lagrange32_dot2_pair).  A sub-block's h
// window is located from the same FP32 positions its samples use (the
// retarded index is monotonic in the sample) and staged as interleaved pairs.
// ---------------------------------------------------------------------------
constexpr int kLgSub = 2 * kTile;      // samples per sub-block
constexpr int kLgWin = kLgSub + 512;   // staged (h+, hx) pairs per sub-block
constexpr int kLgMaxSub = 4;           // sub-blocks per group (groups of up to 8 tiles)

struct LinksGroupSmem {
    TileGeo g;
    float2 win[kLgWin];
    int64_t J[12];
    float f[12];
    Cubic dd[12];
    float dk[6][3];
    Cubic dn[6][3];
    int64_t wlo[kLgMaxSub];
    int wlen[kLgMaxSub];
    int64_t jends[kLgMaxSub][24];
    float inv_half, inv_dt;
};

// Position of block offset dm on the h grid: integer part jp, fraction fp.
__device__ __forceinline__ void lg_pos(const LinksArgs& a, int dm, int& jp, float& fp)
{
    if (a.hm.unit_rho) {
        jp = dm;
        fp = 0.f;
    } else {
        const double P = (double)dm * a.hm.rho;
        const double fl = floor(P);
        jp = (int)fl;
        fp = (float)(P - fl);
    }
}

// Retarded stencil centre (relative to J[lt]) and fraction of link-time lt.
__device__ __forceinline__ void lg_locate(const LinksGroupSmem& s, int lt, float u, int jp, float fp, int& jr,
                                          float& eps)
{
    const float v = (fp + s.f[lt]) - s.dd[lt](u) * s.inv_dt;
    const float fv = floorf(v);
    jr = jp + (int)fv;
    eps = v - fv;
}

// The nt (<= G) tiles from tile t0 of a group of G tiles (centre
// t0 kTile + G kTile / 2): links of samples in [a.i_begin, a.i_end) stored to
// a.y[li * a.ny + i - a.y0].  Every thread of the block must call it; it
// synchronises and leaves the shared memory free.
static __device__ void links_group(const LinksArgs& a, int64_t t0, int nt, int G, LinksGroupSmem& s)
{
    const int t = threadIdx.x;
    const int64_t ic = t0 * kTile + (int64_t)G * kTile / 2;
    const float* __restrict__ hp = (const float*)a.hp;
    const float* __restrict__ hc = (const float*)a.hc;
    float* __restrict__ y = (float*)a.y;
    tile_geo_load(s.g, a.tab, ic, a.sky);   // ends with a block barrier
    const TileGeo& g = s.g;
    if (t == 45) {
        s.inv_half = (float)(2.0 / a.tab.S);
        s.inv_dt = (float)(1.0 / a.hm.dt_in);
    }
    if (t >= 32 && t < 44) {
        // link-time lt = 2 li + {0: sender end T_l + k.R_s/c, 1: receiver end k.R_r/c}
        const int lt = t - 32, li = lt >> 1;
        const int rs = (lt & 1) ? kRowKR + link_receiver(li) : kRowKR + link_sender(li);
        double dc = g.b[rs][0];
        Cubic cv = tg_cubic(g, rs);
        if (!(lt & 1)) {
            dc += g.b[kQT + li][0];
            const Cubic ct = tg_cubic(g, kQT + li);
            cv.c1 += ct.c1;
            cv.c2 += ct.c2;
            cv.c3 += ct.c3;
        }
        int64_t j;
        double eps;
        split_f64(a.hm, ic, dc, j, eps);
        s.J[lt] = j;
        s.f[lt] = (float)eps;
        s.dd[lt] = cv;
    }
    if (t >= 64 && t < 82) {
        const int q = t - 64, li = q / 3, c = q % 3;
        s.dk[li][c] = (float)(g.b[kQN + 3 * li + c][0] - a.sky.k[c]);
        s.dn[li][c] = tg_cubic(g, kQN + 3 * li + c);
    }
    __syncthreads();
    // windows of every sub-block from the link-times at its first and last sample
    const int nsb = (nt + 1) / 2;
    if (t < 24 * nsb) {
        const int sb = t / 24, k = t % 24, lt = k % 12;
        const int64_t i0 = (t0 + 2 * sb) * (int64_t)kTile;
        const int last = (2 * sb + 1 < nt ? kLgSub : kTile) - 1;
        const int dm = (int)(i0 - ic) + (k < 12 ? 0 : last);
        int jp, jr;
        float fp, eps;
        lg_pos(a, dm, jp, fp);
        lg_locate(s, lt, (float)dm * s.inv_half, jp, fp, jr, eps);
        s.jends[sb][k] = s.J[lt] + jr;
    }
    __syncthreads();
    if (t < nsb) {
        int64_t lo = s.jends[t][0], hi = s.jends[t][0];
        for (int k = 1; k < 24; ++k) {
            lo = s.jends[t][k] < lo ? s.jends[t][k] : lo;
            hi = s.jends[t][k] > hi ? s.jends[t][k] : hi;
        }
        s.wlo[t] = lo - 15 - 3;
        const int64_t len = (hi + 16 + 3) - s.wlo[t] + 1;
        s.wlen[t] = len <= kLgWin ? (int)len : 0;
    }
    __syncthreads();
    const float c2 = a.sky.c2f, s2 = a.sky.s2f;
    for (int sb = 0; sb < nsb; ++sb) {
        const int64_t i0 = (t0 + 2 * sb) * (int64_t)kTile;
        const int64_t wlo = s.wlo[sb];
        const int wlen = s.wlen[sb];
        if (sb > 0) __syncthreads();   // the previous sub-block's readers of the window are done
        for (int k = t; k < wlen; k += kTile) {
            const int64_t idx = wlo + k;
            const bool in = idx >= 0 && idx < a.hm.n_in;
            s.win[k] = make_float2(in ? hp[idx] : 0.f, in ? hc[idx] : 0.f);
        }
        __syncthreads();
        // samples i0 + t and i0 + kTile + t
        const int dm0 = (int)(i0 - ic) + t, dm1 = dm0 + kTile;
        const float u0 = (float)dm0 * s.inv_half, u1 = (float)dm1 * s.inv_half;
        int jp0, jp1;
        float fp0, fp1;
        lg_pos(a, dm0, jp0, fp0);
        lg_pos(a, dm1, jp1, fp1);
        auto interp2 = [&](int lt, float2& oa, float2& ob) {
            int ja, jb;
            float ea, eb;
            lg_locate(s, lt, u0, jp0, fp0, ja, ea);
            lg_locate(s, lt, u1, jp1, fp1, jb, eb);
            if (wlen > 0) {
                // every stencil of the sub-block lies in its window; the clamp
                // keeps reads in bounds
                const int rel = (int)(s.J[lt] - wlo) - 15;
                const int ba = min(max(rel + ja, 0), wlen - 32);
                const int bb = min(max(rel + jb, 0), wlen - 32);
                lagrange32_dot2_pair(make_float2(ea, eb), s.win + ba, s.win + bb, oa, ob);
            } else {
                oa = links_interp_global_f32(hp, hc, a.hm.n_in, s.J[lt] + ja, ea);
                ob = links_interp_global_f32(hp, hc, a.hm.n_in, s.J[lt] + jb, eb);
            }
        };
        // receiver ends: the two links into a spacecraft share k.R_r/c (links 3, 0, 1
        // carry the receivers 0, 1, 2)
        float2 ra[3], rb[3];
        interp2(2 * 3 + 1, ra[0], rb[0]);
        interp2(2 * 0 + 1, ra[1], rb[1]);
        interp2(2 * 1 + 1, ra[2], rb[2]);
        const int64_t ia = i0 + t, ib = ia + kTile;
        // the second sample exists only if the sub-block has its second tile in this group
        const bool va = ia >= a.i_begin && ia < a.i_end;
        const bool vb = 2 * sb + 1 < nt && ib >= a.i_begin && ib < a.i_end;
#pragma unroll 1
        for (int li = 0; li < 6; ++li) {
            float2 sa, sbv;
            interp2(2 * li, sa, sbv);
            const int r = link_receiver(li);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float u = q ? u1 : u0;
                float d[3], dd = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    d[c] = s.dk[li][c] + s.dn[li][c](u);
                    dd = fmaf(d[c], d[c], dd);
                }
                const float un = a.sky.uf[0] * d[0] + a.sky.uf[1] * d[1] + a.sky.uf[2] * d[2];
                const float vn = a.sky.vf[0] * d[0] + a.sky.vf[1] * d[1] + a.sky.vf[2] * d[2];
                const float xp = un * un - vn * vn, xc = 2.f * un * vn;
                const float rdd = 1.f / dd;
                const float Fp = (xp * c2 + xc * s2) * rdd, Fc = (xc * c2 - xp * s2) * rdd;
                const float2 hs = q ? sbv : sa, hr = q ? rb[r] : ra[r];
                const float v = Fp * (hs.x - hr.x) + Fc * (hs.y - hr.y);
                const int64_t i = q ? ib : ia;
                if (q ? vb : va) y[(int64_t)li * a.ny + (i - a.y0)] = dd >= 2e-12f ? v : 0.f;
            }
        }
    }
    __syncthreads();   // the shared memory is free for the caller
}


}  // namespace lisa
