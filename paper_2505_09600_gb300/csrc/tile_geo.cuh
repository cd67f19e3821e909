// Tile-local orbit geometry: the segment polynomial of every orbit quantity
// re-expanded (Taylor shift, FP64) around the tile's centre sample, plus the
// source projections k.R_s/c.  One instance lives in shared memory per CTA.
#pragma once

#include "lisa_common.cuh"

namespace lisa {

constexpr int kRowKR = kNQ;       // rows 33..35: k.R_s / c
constexpr int kRows = kNQ + 3;

struct TileGeo {
    double b[kRows][8];
};

// Fill g for the tile whose centre sample is ic.  Must be called by every
// thread of the block (contains __syncthreads).  Requires blockDim.x >= 36.
__device__ __forceinline__ void tile_geo_load(TileGeo& g, const SegTable& tab, int64_t ic, const SkyDev& sky)
{
    int64_t s = ic / tab.S;
    if (s >= tab.nseg) s = tab.nseg - 1;
    if (s < 0) s = 0;
    const double half = 0.5 * tab.S;
    const double xc = ((double)(ic - s * tab.S) - half) / half;
    const int q = threadIdx.x;
    if (q < kNQ) {
        double b[7];
        taylor_shift7(tab.coef + (s * kNQ + q) * kNC, xc, b);
#pragma unroll
        for (int p = 0; p < 7; ++p) g.b[q][p] = b[p];
        g.b[q][7] = 0.0;
    }
    __syncthreads();
    if (q < 3 * 8) {
        const int sc = q / 8, p = q % 8;
        g.b[kRowKR + sc][p] = (sky.k[0] * g.b[kQR + 3 * sc][p] + sky.k[1] * g.b[kQR + 3 * sc + 1][p]
                               + sky.k[2] * g.b[kQR + 3 * sc + 2][p]) / kC;
    }
    __syncthreads();
}

__device__ __forceinline__ double tg_eval(const TileGeo& g, int row, double u) { return horner_d<7>(g.b[row], u); }

// In-tile variation (value minus the centre value) as an FP32 cubic: the
// omitted u^4.. terms are < 1e-12 s for any delay over a 256-sample tile.
struct Cubic {
    float c1, c2, c3;
    __device__ __forceinline__ float operator()(float u) const { return u * fmaf(u, fmaf(u, c3, c2), c1); }
};

__device__ __forceinline__ Cubic tg_cubic(const TileGeo& g, int row)
{
    return Cubic{(float)g.b[row][1], (float)g.b[row][2], (float)g.b[row][3]};
}

}  // namespace lisa
