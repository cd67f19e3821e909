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
#include "links_group.cuh"

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
    links_sample<MIXED>(a, g, ic, i, s, (Real*)a.y + (i - a.y0), a.ny);
}

// FP64 form on short ranges (a hybrid's full part covers a few tiles): the
// six links of a tile and its samples are split over 6 x parts CTAs, CTA
// (tile, li * parts + part) holding link li of kTile / parts samples.
__global__ void __launch_bounds__(kTile) links_full_kernel_f64_split(LinksArgs a, int parts)
{
    __shared__ TileGeo g;
    __shared__ LinksTile<false> s;
    const int64_t i0 = (a.tile0 + blockIdx.x) * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    tile_geo_load(g, a.tab, ic, a.sky);
    links_tile_prologue<false>(a, g, ic, i0, i0 + kTile - 1, s);
    const int li = blockIdx.y / parts, part = blockIdx.y % parts;
    const int per = kTile / parts;
    if ((int)threadIdx.x >= per) return;
    const int64_t i = i0 + (int64_t)part * per + threadIdx.x;
    if (i < a.i_begin || i >= a.i_end) return;
    const double u = (double)(i - ic) / (0.5 * a.tab.S);
    double kR[3];
#pragma unroll
    for (int sc = 0; sc < 3; ++sc) kR[sc] = tg_eval(g, kRowKR + sc, u);
    ((double*)a.y)[(int64_t)li * a.ny + (i - a.y0)] = link_value_f64(a, g, u, i, s, li, kR);
}

__global__ void __launch_bounds__(kTile, 3) links_group_kernel(LinksArgs a, int64_t tile_end, int G)
{
    __shared__ LinksGroupSmem s;
    const int64_t t0 = a.tile0 + (int64_t)blockIdx.x * G;
    const int nt = (int)(tile_end - t0 < G ? tile_end - t0 : G);
    links_group(a, t0, nt, G, s);
}

int launch_links_full(const SegTable& tab, const SkyDev& sky, const lisa_grid& hg, const void* hp, const void* hc,
                      int precision, const lisa_grid& yg, void* y, int64_t i_begin, int64_t i_end, cudaStream_t st,
                      int64_t y0)
{
    if (i_end <= i_begin) return LISA_OK;
    LinksArgs a;
    a.tab = tab;
    a.sky = sky;
    a.hm = make_grid_map(yg, hg);
    a.hp = hp;
    a.hc = hc;
    a.y = y;
    a.y0 = y0;
    a.ny = yg.n - y0;
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
    } else if (tiles < 2 * 152) {
        // split the links (and, for very short ranges, the samples) so that
        // the launch fills about two CTAs per SM
        const int parts = tiles * 6 >= 2 * 152 ? 1 : tiles * 12 >= 2 * 152 ? 2 : 4;
        links_full_kernel_f64_split<<<dim3((unsigned)tiles, 6u * parts), kTile, 0, st>>>(a, parts);
    } else {
        links_full_kernel<false><<<(unsigned)tiles, kTile, 0, st>>>(a);
    }
    prof_after(st);
    return cuda_status(cudaGetLastError(), "links_full_kernel launch");
}

}  // namespace lisa
