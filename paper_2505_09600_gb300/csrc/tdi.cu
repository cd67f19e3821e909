// Michelson TDI 1.5 / 2.0 (Sec. II B, Eqs. X1.5, X2.0), Y and Z by cyclic
// permutation, optional A, E, T, optional hybrid sigmoid weight.
//
// Each term is a signed link series delayed by an ordered list of light
// times.  The lists follow the operator form
//   X1.5 = (A-1)a + (1-B)b,  X2.0 = (A-1+AB-BAA)a + (1-B-BA+ABB)b,
//   A = D_-2 D_2, B = D_3 D_-3, a = y_231 + D_3 y_1-32, b = y_3-21 + D_-2 y_123,
// whose expansion gives every delay sum and sign of Eqs. X1.5, X2.0.  FROZEN
// sums the light times at the output time; NESTED applies them in order,
// each at its own retarded time.
//
// One CTA per tile of kTile output samples, one thread per sample.  The six
// link series are staged in shared memory over the window the tile's delays
// (0 .. 7 T_max) can reach.
#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "tile_geo.cuh"

namespace lisa {

constexpr int kWinY = kTile + 256;

struct TdiTerm {
    int sign, link, nd;
    int d[8];
};

__constant__ TdiTerm c_terms[16] = {
    {+1, 5, 3, {3, 2, 4}},              {-1, 5, 1, {4}},
    {+1, 4, 2, {3, 2}},                 {-1, 4, 0, {0}},
    {+1, 2, 1, {3}},                    {-1, 2, 3, {4, 5, 3}},
    {+1, 3, 0, {0}},                    {-1, 3, 2, {4, 5}},
    {+1, 5, 5, {3, 2, 4, 5, 4}},        {-1, 5, 7, {4, 5, 3, 2, 3, 2, 4}},
    {+1, 4, 4, {3, 2, 4, 5}},           {-1, 4, 6, {4, 5, 3, 2, 3, 2}},
    {+1, 2, 7, {3, 2, 4, 5, 4, 5, 3}},  {-1, 2, 5, {4, 5, 3, 2, 3}},
    {+1, 3, 6, {3, 2, 4, 5, 4, 5}},     {-1, 3, 4, {4, 5, 3, 2}},
};
__constant__ int c_cyc[3][6] = {{0, 1, 2, 3, 4, 5}, {2, 3, 4, 5, 0, 1}, {4, 5, 0, 1, 2, 3}};

struct TdiArgs {
    SegTable tab;
    GridMap ym;
    const void* y;
    int64_t ny;
    void* xyz;
    int64_t nout;
    int nterm, mode, channels;
    int64_t i_begin, i_end, tile0;
    BlendSpec bl;
    double t0_out, dt_out;
};

template <typename Real>
__device__ __forceinline__ Real interp_one(const Real* win, int64_t wlo, int wlen, const Real* __restrict__ yg,
                                           int64_t n, int64_t j, Real eps)
{
    if (eps == Real(0)) {
        const int64_t o = j - wlo;
        if (o >= 0 && o < wlen) return win[o];
        return (j >= 0 && j < n) ? yg[j] : Real(0);
    }
    Real w[32];
    lagrange32_weights(eps, w);
    Real acc = Real(0);
    const int64_t base = j - 15 - wlo;
    if (base >= 0 && base + 32 <= wlen) {
        const Real* p = win + base;
#pragma unroll
        for (int k = 0; k < 32; ++k) acc = fma(w[k], p[k], acc);
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int64_t idx = j - 15 + k;
            if (idx >= 0 && idx < n) acc = fma(w[k], yg[idx], acc);
        }
    }
    return acc;
}

// Epilogue shared by the full and LFA channel kernels: optional AET, optional
// sigmoid weight, optional accumulation onto the existing output.
template <typename Real>
__device__ __forceinline__ void store_channels(Real X, Real Y, Real Z, int channels, const BlendSpec& bl,
                                               double t0, double dt, int64_t i, Real* __restrict__ out, int64_t n)
{
    Real o0 = X, o1 = Y, o2 = Z;
    if (channels == LISA_AET) {
        o0 = (Z - X) * Real(0.70710678118654752440);
        o1 = (X - Real(2) * Y + Z) * Real(0.40824829046386301637);
        o2 = (X + Y + Z) * Real(0.57735026918962576451);
    }
    if (bl.enabled) {
        const double ti = t0 + (double)i * dt;
        const double arg = bl.eps * (ti - bl.t_hyb) / bl.sigma;
        Real wgt;
        if constexpr (sizeof(Real) == 8) wgt = 1.0 / (1.0 + exp(arg));
        else wgt = 1.f / (1.f + expf((float)arg));
        o0 *= wgt;
        o1 *= wgt;
        o2 *= wgt;
        if (i >= bl.acc_begin && i < bl.acc_end) {
            o0 += out[i];
            o1 += out[n + i];
            o2 += out[2 * n + i];
        }
    }
    out[i] = o0;
    out[n + i] = o1;
    out[2 * n + i] = o2;
}

template <bool MIXED>
__global__ void __launch_bounds__(kTile) tdi_kernel(TdiArgs a)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    __shared__ TileGeo g;
    __shared__ Real win[6][kWinY];
    __shared__ int64_t s_wlo;
    __shared__ int s_wlen;
    __shared__ double s_Tc[6];
    // mixed, frozen: per (channel, term) centre split and in-tile cubic
    __shared__ int64_t s_J[48];
    __shared__ float s_f[48];
    __shared__ Cubic s_dD[48];

    const Real* __restrict__ yg = (const Real*)a.y;
    Real* __restrict__ out = (Real*)a.xyz;
    const int64_t i0 = (a.tile0 + blockIdx.x) * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    const double half = 0.5 * a.tab.S;
    const int t = threadIdx.x;
    tile_geo_load(g, a.tab, ic, SkyDev{});

    if (t < 6) s_Tc[t] = g.b[kQT + t][0];
    if constexpr (MIXED) {
        if (a.mode == LISA_FROZEN && t >= 64 && t < 64 + 3 * a.nterm) {
            const int w = t - 64, ch = w / a.nterm, q = w % a.nterm;
            const TdiTerm& tm = c_terms[q];
            double Dc = 0.0;
            Cubic cv{0.f, 0.f, 0.f};
            for (int k = 0; k < tm.nd; ++k) {
                const int row = kQT + c_cyc[ch][tm.d[k]];
                Dc += g.b[row][0];
                const Cubic cr = tg_cubic(g, row);
                cv.c1 += cr.c1; cv.c2 += cr.c2; cv.c3 += cr.c3;
            }
            int64_t j;
            double eps;
            split_f64(a.ym, ic, Dc, j, eps);
            s_J[w] = j;
            s_f[w] = (float)eps;
            s_dD[w] = cv;
        }
    }
    __syncthreads();
    if (t == 0) {
        // largest delay of any term: up to 7 light times, +1 s of margin
        double Tmax = 0.0;
        for (int li = 0; li < 6; ++li) {
            const double a0 = tg_eval(g, kQT + li, (double)(i0 - ic) / half);
            const double a1 = tg_eval(g, kQT + li, (double)(i0 + kTile - 1 - ic) / half);
            Tmax = fmax(Tmax, fmax(a0, a1));
        }
        const double Dmax = (a.nterm == 16 ? 7.0 : 3.0) * Tmax + 1.0;
        int64_t jlo, jhi;
        double e;
        split_f64(a.ym, i0, Dmax, jlo, e);
        split_f64(a.ym, i0 + kTile - 1, -1.0, jhi, e);
        s_wlo = jlo - 15 - 2;
        const int64_t len = (jhi + 16 + 2) - s_wlo + 1;
        s_wlen = len <= kWinY ? (int)len : 0;
    }
    __syncthreads();
    const int64_t wlo = s_wlo;
    const int wlen = s_wlen;
    for (int k = t; k < 6 * wlen; k += blockDim.x) {
        const int li = k / wlen, o = k % wlen;
        const int64_t idx = wlo + o;
        win[li][o] = (idx >= 0 && idx < a.ym.n_in) ? yg[(int64_t)li * a.ny + idx] : Real(0);
    }
    __syncthreads();

    const int64_t i = i0 + t;
    if (i < a.i_begin || i >= a.i_end) return;

    Real acc[3] = {Real(0), Real(0), Real(0)};
    if (!MIXED || a.mode == LISA_NESTED) {
        const double u = (double)(i - ic) / half;
        double T[6];
#pragma unroll
        for (int li = 0; li < 6; ++li) T[li] = tg_eval(g, kQT + li, u);
#pragma unroll 1
        for (int ch = 0; ch < 3; ++ch) {
#pragma unroll 1
            for (int q = 0; q < a.nterm; ++q) {
                const TdiTerm& tm = c_terms[q];
                double D = 0.0;
                for (int k = 0; k < tm.nd; ++k) {
                    const int li = c_cyc[ch][tm.d[k]];
                    if (a.mode == LISA_NESTED) {
                        D += tg_eval(g, kQT + li, u - D / (a.dt_out * half));
                    } else {
                        double Tl = T[0];
                        for (int r = 1; r < 6; ++r) Tl = (li == r) ? T[r] : Tl;
                        D += Tl;
                    }
                }
                int64_t j;
                double eps;
                split_f64(a.ym, i, D, j, eps);
                const int ls = c_cyc[ch][tm.link];
                const Real v = interp_one<Real>(win[ls], wlo, wlen, yg + (int64_t)ls * a.ny, a.ym.n_in, j, (Real)eps);
                acc[ch] += (tm.sign > 0) ? v : -v;
            }
        }
    } else if constexpr (MIXED) {
        const float u = (float)(i - ic) / (float)half;
        int64_t jp;
        float fp;
        if (a.ym.unit_rho) {
            jp = i - ic;
            fp = 0.f;
        } else {
            const double P = (double)(i - ic) * a.ym.rho;
            const double fl = floor(P);
            jp = (int64_t)fl;
            fp = (float)(P - fl);
        }
        const float inv_dt = (float)(1.0 / a.ym.dt_in);
#pragma unroll 1
        for (int ch = 0; ch < 3; ++ch) {
#pragma unroll 1
            for (int q = 0; q < a.nterm; ++q) {
                const int w = ch * a.nterm + q;
                const float v = (fp + s_f[w]) - s_dD[w](u) * inv_dt;
                const float fv = floorf(v);
                const int64_t j = s_J[w] + jp + (int64_t)fv;
                const float eps = v - fv;
                const TdiTerm& tm = c_terms[q];
                const int ls = c_cyc[ch][tm.link];
                const float val = interp_one<float>(win[ls], wlo, wlen, yg + (int64_t)ls * a.ny, a.ym.n_in, j, eps);
                acc[ch] += (tm.sign > 0) ? val : -val;
            }
        }
    }
    store_channels<Real>(acc[0], acc[1], acc[2], a.channels, a.bl, a.t0_out, a.dt_out, i, out, a.nout);
}

int launch_tdi(const SegTable& tab, const lisa_grid& yg, const void* y, int precision, int gen, int mode, int channels,
               const lisa_grid& og, void* xyz, int64_t i_begin, int64_t i_end, const BlendSpec& bl, cudaStream_t st)
{
    if (i_end <= i_begin) return LISA_OK;
    TdiArgs a;
    a.tab = tab;
    a.ym = make_grid_map(og, yg);
    a.y = y;
    a.ny = yg.n;
    a.xyz = xyz;
    a.nout = og.n;
    a.nterm = (gen == LISA_TDI20) ? 16 : 8;
    a.mode = mode;
    a.channels = channels;
    a.i_begin = i_begin;
    a.i_end = i_end;
    a.tile0 = i_begin / kTile;
    a.bl = bl;
    a.t0_out = og.t0;
    a.dt_out = og.dt;
    const int64_t tiles = (i_end - 1) / kTile - a.tile0 + 1;
    prof_before(precision == LISA_MIXED ? "tdi_mixed" : "tdi_f64", st);
    if (precision == LISA_MIXED) tdi_kernel<true><<<(unsigned)tiles, kTile, 0, st>>>(a);
    else tdi_kernel<false><<<(unsigned)tiles, kTile, 0, st>>>(a);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "tdi_kernel launch");
}

}  // namespace lisa
