// Full single-link response (Sec. II A-B, Eqs. H, yslr, delta_s, delta_r):
//   y_l(t) = [H_l(t - delta_s) - H_l(t - delta_r)] / (2 (1 - k.n_l)),
//   H_l = xi+_l h+SSB + xix_l hxSSB,  delta_s = T_l + k.R_s/c, delta_r = k.R_r/c.
//
// One CTA computes a tile of kTile consecutive output samples, one thread per
// sample, all six links.  The h+/hx window that the tile's twelve retarded
// times can reach (tile length + ~17 s of link spread + 32-point stencil) is
// staged once in shared memory as interleaved (h+, hx) pairs, so each
// interpolation reads 32 consecutive pairs that neighbouring lanes share.
//
// The polarisation rotation and the antenna patterns are folded into two
// factors per link, using 2(1 - k.n) = |n - k|^2 and u.n = u.(n - k),
// v.n = v.(n - k) (u, v are orthogonal to k):
//   y_l = F+ [h+(t-ds) - h+(t-dr)] + Fx [hx(t-ds) - hx(t-dr)],
//   F+ = (xi+ cos2psi + xix sin2psi)/|n-k|^2,  Fx = (xix cos2psi - xi+ sin2psi)/|n-k|^2,
// which stays well conditioned when the source lies close to a link
// (|F| <= 1).  Links with |n - k|^2 < 2e-12 are set to zero.
#include "links_tile.cuh"

#ifndef LISA_LINKS_GROUPED
#define LISA_LINKS_GROUPED 1   // mixed form: groups of tiles around one FP64 set-up, paired samples
#endif

namespace lisa {

template <bool MIXED>
__global__ void __launch_bounds__(kTile) links_full_kernel(LinksArgs a)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    __shared__ TileGeo g;
    __shared__ LinksTile<MIXED> s;
    const int64_t i0 = (a.tile0 + blockIdx.x) * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    tile_geo_load(g, a.tab, ic, a.sky);
    links_tile_prologue<MIXED>(a, g, ic, i0, i0 + kTile - 1, s);
    const int64_t i = i0 + threadIdx.x;
    if (i < a.i_begin || i >= a.i_end) return;
    links_sample<MIXED>(a, g, ic, i, s, (Real*)a.y + i, a.ny);
}

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

__global__ void __launch_bounds__(kTile, 3) links_group_kernel(LinksArgs a, int64_t tile_end, int G)
{
    __shared__ LinksGroupSmem s;
    const int t = threadIdx.x;
    const int64_t t0 = a.tile0 + (int64_t)blockIdx.x * G;
    const int nt = (int)(tile_end - t0 < G ? tile_end - t0 : G);
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
                if (q ? vb : va) y[(int64_t)li * a.ny + i] = dd >= 2e-12f ? v : 0.f;
            }
        }
    }
}

int launch_links_full(const SegTable& tab, const SkyDev& sky, const lisa_grid& hg, const void* hp, const void* hc,
                      int precision, const lisa_grid& yg, void* y, int64_t i_begin, int64_t i_end, cudaStream_t st)
{
    if (i_end <= i_begin) return LISA_OK;
    LinksArgs a;
    a.tab = tab;
    a.sky = sky;
    a.hm = make_grid_map(yg, hg);
    a.hp = hp;
    a.hc = hc;
    a.y = y;
    a.ny = yg.n;
    a.i_begin = i_begin;
    a.i_end = i_end;
    a.tile0 = i_begin / kTile;
    const int64_t tiles = (i_end - 1) / kTile - a.tile0 + 1;
    prof_before(precision == LISA_MIXED ? "links_full_mixed" : "links_full_f64", st);
    if (precision == LISA_MIXED) {
#if LISA_LINKS_GROUPED
        // groups as long as the span bound allows, shorter when the range is
        // small: at least one wave of CTAs (152 SMs x 3)
        int G = lfa_group_host(yg.dt);
        const int64_t per_wave = tiles / (152 * 3);
        if (per_wave < G) G = per_wave > 1 ? (int)per_wave : 1;
        const int64_t tile_end = a.tile0 + tiles;
        links_group_kernel<<<(unsigned)((tiles + G - 1) / G), kTile, 0, st>>>(a, tile_end, G);
#else
        links_full_kernel<true><<<(unsigned)tiles, kTile, 0, st>>>(a);
#endif
    } else {
        links_full_kernel<false><<<(unsigned)tiles, kTile, 0, st>>>(a);
    }
    prof_after(st);
    return cuda_status(cudaGetLastError(), "links_full_kernel launch");
}

}  // namespace lisa
