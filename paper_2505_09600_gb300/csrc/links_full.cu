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
#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "tile_geo.cuh"

namespace lisa {

constexpr int kWinMax = kTile + 768;

template <typename Real>
struct Pair;
template <>
struct Pair<double> { using T = double2; };
template <>
struct Pair<float> { using T = float2; };

struct LinksArgs {
    SegTable tab;
    SkyDev sky;
    GridMap hm;
    const void* hp;
    const void* hc;
    void* y;
    int64_t ny;
    int64_t i_begin, i_end;
    int64_t tile0;
};

// Interpolate both polarisations at (j, eps) from the staged window, or from
// global memory when the stencil is not inside the window.
template <typename Real>
__device__ __forceinline__ void interp_pair(const typename Pair<Real>::T* win, int64_t wlo, int wlen,
                                            const Real* __restrict__ hp, const Real* __restrict__ hc, int64_t nh,
                                            int64_t j, Real eps, Real& op, Real& oc)
{
    const int64_t base = j - 15 - wlo;
    if (eps == Real(0)) {
        const int64_t o = j - wlo;
        if (o >= 0 && o < wlen) {
            op = win[o].x;
            oc = win[o].y;
        } else {
            op = (j >= 0 && j < nh) ? hp[j] : Real(0);
            oc = (j >= 0 && j < nh) ? hc[j] : Real(0);
        }
        return;
    }
    Real w[32];
    lagrange32_weights(eps, w);
    Real ap = Real(0), ac = Real(0);
    if (base >= 0 && base + 32 <= wlen) {
        const typename Pair<Real>::T* p = win + base;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const typename Pair<Real>::T v = p[k];
            ap = fma(w[k], v.x, ap);
            ac = fma(w[k], v.y, ac);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int64_t idx = j - 15 + k;
            if (idx >= 0 && idx < nh) {
                ap = fma(w[k], hp[idx], ap);
                ac = fma(w[k], hc[idx], ac);
            }
        }
    }
    op = ap;
    oc = ac;
}

template <bool MIXED>
__global__ void __launch_bounds__(kTile) links_full_kernel(LinksArgs a)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    using Real2 = typename Pair<Real>::T;
    __shared__ TileGeo g;
    __shared__ Real2 win[kWinMax];
    __shared__ int64_t jends[24];
    __shared__ int64_t s_wlo;
    __shared__ int s_wlen;
    // mixed-precision per-tile delay data (12 link-times: li*2 + {0: sender, 1: receiver})
    __shared__ int64_t s_J[12];
    __shared__ float s_f[12];
    __shared__ Cubic s_dd[12];
    __shared__ float s_dk[6][3];
    __shared__ Cubic s_dn[6][3];

    const Real* __restrict__ hp = (const Real*)a.hp;
    const Real* __restrict__ hc = (const Real*)a.hc;
    Real* __restrict__ y = (Real*)a.y;

    const int64_t i0 = (a.tile0 + blockIdx.x) * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    const double half = 0.5 * a.tab.S;
    tile_geo_load(g, a.tab, ic, a.sky);

    // --- window of h reachable by this tile -------------------------------
    const int t = threadIdx.x;
    if (t < 24) {
        const int end = t / 12, lt = t % 12, li = lt >> 1;
        const int64_t ie = end ? i0 + kTile - 1 : i0;
        const double u = (double)(ie - ic) / half;
        const double d = (lt & 1) ? tg_eval(g, kRowKR + link_receiver(li), u)
                                  : tg_eval(g, kQT + li, u) + tg_eval(g, kRowKR + link_sender(li), u);
        int64_t j;
        double eps;
        split_f64(a.hm, ie, d, j, eps);
        jends[t] = j;
    }
    if constexpr (MIXED) {
        if (t >= 32 && t < 44) {
            const int lt = t - 32, li = lt >> 1;
            const int rs = (lt & 1) ? kRowKR + link_receiver(li) : kRowKR + link_sender(li);
            double dc = g.b[rs][0];
            Cubic cv = tg_cubic(g, rs);
            if (!(lt & 1)) {
                dc += g.b[kQT + li][0];
                const Cubic ct = tg_cubic(g, kQT + li);
                cv.c1 += ct.c1; cv.c2 += ct.c2; cv.c3 += ct.c3;
            }
            int64_t j;
            double eps;
            split_f64(a.hm, ic, dc, j, eps);
            s_J[lt] = j;
            s_f[lt] = (float)eps;
            s_dd[lt] = cv;
        }
        if (t >= 64 && t < 82) {
            const int q = t - 64, li = q / 3, c = q % 3;
            s_dk[li][c] = (float)(g.b[kQN + 3 * li + c][0] - a.sky.k[c]);
            s_dn[li][c] = tg_cubic(g, kQN + 3 * li + c);
        }
    }
    __syncthreads();
    if (t == 0) {
        int64_t lo = jends[0], hi = jends[0];
        for (int k = 1; k < 24; ++k) {
            lo = jends[k] < lo ? jends[k] : lo;
            hi = jends[k] > hi ? jends[k] : hi;
        }
        s_wlo = lo - 15 - 3;
        const int64_t len = (hi + 16 + 3) - s_wlo + 1;
        s_wlen = len <= kWinMax ? (int)len : 0;
    }
    __syncthreads();
    const int64_t wlo = s_wlo;
    const int wlen = s_wlen;
    for (int k = t; k < wlen; k += blockDim.x) {
        const int64_t idx = wlo + k;
        Real2 v;
        v.x = (idx >= 0 && idx < a.hm.n_in) ? hp[idx] : Real(0);
        v.y = (idx >= 0 && idx < a.hm.n_in) ? hc[idx] : Real(0);
        win[k] = v;
    }
    __syncthreads();

    const int64_t i = i0 + t;
    if (i < a.i_begin || i >= a.i_end) return;

    const Real c2 = (Real)a.sky.c2p, s2 = (Real)a.sky.s2p;
    const Real ku[3] = {(Real)a.sky.u[0], (Real)a.sky.u[1], (Real)a.sky.u[2]};
    const Real kv[3] = {(Real)a.sky.v[0], (Real)a.sky.v[1], (Real)a.sky.v[2]};

    if constexpr (!MIXED) {
        const double u = (double)(i - ic) / half;
        double kR[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) kR[s] = tg_eval(g, kRowKR + s, u);
#pragma unroll 1
        for (int li = 0; li < 6; ++li) {
            double d[3], dd = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                d[c] = tg_eval(g, kQN + 3 * li + c, u) - a.sky.k[c];
                dd = fma(d[c], d[c], dd);
            }
            double yv = 0.0;
            if (dd >= 2e-12) {
                const double un = ku[0] * d[0] + ku[1] * d[1] + ku[2] * d[2];
                const double vn = kv[0] * d[0] + kv[1] * d[1] + kv[2] * d[2];
                const double xp = un * un - vn * vn, xc = 2.0 * un * vn;
                const double Fp = (xp * c2 + xc * s2) / dd, Fc = (xc * c2 - xp * s2) / dd;
                const double ds = tg_eval(g, kQT + li, u) + kR[link_sender(li)];
                const double dr = kR[link_receiver(li)];
                int64_t js, jr;
                double es, er;
                split_f64(a.hm, i, ds, js, es);
                split_f64(a.hm, i, dr, jr, er);
                double ps, cs, pr, cr;
                interp_pair<double>(win, wlo, wlen, hp, hc, a.hm.n_in, js, es, ps, cs);
                interp_pair<double>(win, wlo, wlen, hp, hc, a.hm.n_in, jr, er, pr, cr);
                yv = Fp * (ps - pr) + Fc * (cs - cr);
            }
            y[(int64_t)li * a.ny + i] = yv;
        }
    } else {
        const float u = (float)(i - ic) / (float)half;
        // integer / fractional split of (i - ic) * rho, shared by all link-times
        int64_t jp;
        float fp;
        if (a.hm.unit_rho) {
            jp = i - ic;
            fp = 0.f;
        } else {
            const double P = (double)(i - ic) * a.hm.rho;
            const double fl = floor(P);
            jp = (int64_t)fl;
            fp = (float)(P - fl);
        }
        const float inv_dt = (float)(1.0 / a.hm.dt_in);
#pragma unroll 1
        for (int li = 0; li < 6; ++li) {
            float d[3], dd = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                d[c] = s_dk[li][c] + s_dn[li][c](u);
                dd = fmaf(d[c], d[c], dd);
            }
            float yv = 0.f;
            if (dd >= 2e-12f) {
                const float un = ku[0] * d[0] + ku[1] * d[1] + ku[2] * d[2];
                const float vn = kv[0] * d[0] + kv[1] * d[1] + kv[2] * d[2];
                const float xp = un * un - vn * vn, xc = 2.f * un * vn;
                const float rdd = 1.f / dd;
                const float Fp = (xp * c2 + xc * s2) * rdd, Fc = (xc * c2 - xp * s2) * rdd;
                float vals[4];
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    const int lt = 2 * li + w;
                    const float v = (fp + s_f[lt]) - s_dd[lt](u) * inv_dt;
                    const float fv = floorf(v);
                    const int64_t j = s_J[lt] + jp + (int64_t)fv;
                    const float eps = v - fv;
                    interp_pair<float>(win, wlo, wlen, hp, hc, a.hm.n_in, j, eps, vals[2 * w], vals[2 * w + 1]);
                }
                yv = Fp * (vals[0] - vals[2]) + Fc * (vals[1] - vals[3]);
            }
            y[(int64_t)li * a.ny + i] = yv;
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
    if (precision == LISA_MIXED) links_full_kernel<true><<<(unsigned)tiles, kTile, 0, st>>>(a);
    else links_full_kernel<false><<<(unsigned)tiles, kTile, 0, st>>>(a);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "links_full_kernel launch");
}

}  // namespace lisa
