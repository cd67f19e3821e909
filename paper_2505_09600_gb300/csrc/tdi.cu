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
#include "tdi_tile.cuh"

namespace lisa {

// Mixed frozen form on a common grid: per-link combined filters (tdi_comb.cu).
int launch_tdi_comb(const TdiArgs& a, int64_t tiles, cudaStream_t st);
// FP64 frozen form on a common grid: per-link combined filters (tdi_comb64.cu).
int launch_tdi_comb64(const TdiArgs& a, cudaStream_t st);

#ifndef LISA_TDI_COMB64
#define LISA_TDI_COMB64 1   // FP64 frozen TDI on combined filters (0: the per-term kernels)
#endif

template <bool MIXED>
__global__ void __launch_bounds__(kTile) tdi_kernel(TdiArgs a)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    __shared__ TileGeo g;
    __shared__ TdiTile<MIXED> s;
    const int64_t i0 = (a.tile0 + blockIdx.x) * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    tile_geo_load(g, a.tab, ic, SkyDev{});
    tdi_tile_prologue<MIXED>(a, g, ic, i0, s);
    tdi_fill_global<MIXED>(a, s);
    const int64_t i = i0 + threadIdx.x;
    if (i < a.i_begin || i >= a.i_end) return;
    Real acc[3];
    tdi_sample<MIXED>(a, g, ic, i, s, acc);
    if constexpr (MIXED)
        store_channels_f32(acc[0], acc[1], acc[2], a.channels, a.bl, s.barg_c, s.barg_d, (int)(i - ic), i,
                           (float*)a.xyz, a.nout);
    else
        store_channels<Real>(acc[0], acc[1], acc[2], a.channels, a.bl, a.t0_out, a.dt_out, i, (Real*)a.xyz, a.nout);
}

// FP64 form on short ranges: the TDI sums of one tile are split over
// `split` CTAs of kTile / split samples each (the FP64 pipe of an SM, not its
// threads, bounds the per-tile form, and a hybrid's full part covers only a
// few tiles).  Thread t handles channel t / spc of sample t % spc; the three
// channels meet in shared memory for A/E/T, the blend and the store.
constexpr int kSplitMin = 4;   // spc <= kTile / kSplitMin samples per CTA

__device__ __forceinline__ double tdi_channel_f64(const TdiArgs& a, const TileGeo& g, int64_t ic, int64_t i,
                                                  const TdiTile<false>& s, int ch)
{
    const double* __restrict__ yg = (const double*)a.y;
    const double half = 0.5 * a.tab.S;
    const double u = (double)(i - ic) / half;
    double T[6];
#pragma unroll
    for (int li = 0; li < 6; ++li) T[li] = tg_eval(g, kQT + li, u);
    double acc = 0.0;
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
        const double v = interp_one<double>(s.win[ls], s.wlo, s.wlen, yg ? yg + (int64_t)ls * a.ny : nullptr,
                                            yg ? a.ym.n_in : 0, j, eps);
        acc += (tm.sign > 0) ? v : -v;
    }
    return acc;
}

__global__ void __launch_bounds__(kTile) tdi_kernel_f64_split(TdiArgs a, int spc)
{
    __shared__ TileGeo g;
    __shared__ TdiTile<false> s;
    __shared__ double xs[3][kTile / kSplitMin];
    const int64_t i0 = (a.tile0 + blockIdx.x) * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    tile_geo_load(g, a.tab, ic, SkyDev{});
    tdi_tile_prologue<false>(a, g, ic, i0, s);
    tdi_fill_global<false>(a, s);
    const int t = threadIdx.x;
    const int64_t ib = i0 + (int64_t)blockIdx.y * spc;
    if (t < 3 * spc) {
        const int ch = t / spc;
        const int64_t i = ib + t % spc;
        xs[ch][t % spc] = (i >= a.i_begin && i < a.i_end) ? tdi_channel_f64(a, g, ic, i, s, ch) : 0.0;
    }
    __syncthreads();
    if (t < spc) {
        const int64_t i = ib + t;
        if (i >= a.i_begin && i < a.i_end)
            store_channels<double>(xs[0][t], xs[1][t], xs[2][t], a.channels, a.bl, a.t0_out, a.dt_out, i,
                                   (double*)a.xyz, a.nout);
    }
}

int launch_tdi(const SegTable& tab, const lisa_grid& yg, const void* y, int precision, int gen, int mode, int channels,
               const lisa_grid& og, void* xyz, int64_t i_begin, int64_t i_end, const BlendSpec& bl, cudaStream_t st,
               int64_t y0)
{
    if (i_end <= i_begin) return LISA_OK;
    TdiArgs a;
    a.tab = tab;
    // y holds the link grid's samples [y0, yg.n): the map to it is the map to
    // the whole grid shifted by the integer y0 (exact)
    a.ym = make_grid_map(og, yg);
    a.ym.jb -= y0;
    a.ym.n_in = yg.n - y0;
    a.y = y;
    a.ny = yg.n - y0;
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
    int rc;
    if (precision == LISA_MIXED && mode == LISA_FROZEN && a.ym.unit_rho) {
        rc = launch_tdi_comb(a, tiles, st);
    } else if (LISA_TDI_COMB64 && precision != LISA_MIXED && mode == LISA_FROZEN && a.ym.unit_rho) {
        rc = launch_tdi_comb64(a, st);
    } else {
        if (precision == LISA_MIXED) tdi_kernel<true><<<(unsigned)tiles, kTile, 0, st>>>(a);
        else if (tiles < 2 * 152) {
            // about two CTAs per SM: 4, 8 or 16 CTAs per tile
            const int split = tiles * 4 >= 2 * 152 ? 4 : tiles * 8 >= 2 * 152 ? 8 : 16;
            tdi_kernel_f64_split<<<dim3((unsigned)tiles, (unsigned)split), kTile, 0, st>>>(a, kTile / split);
        }
        else tdi_kernel<false><<<(unsigned)tiles, kTile, 0, st>>>(a);
        rc = cuda_status(cudaGetLastError(), "tdi_kernel launch");
    }
    prof_after(st);
    return rc;
}

}  // namespace lisa
