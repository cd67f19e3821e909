// Mixed frozen TDI on per-link combined filters: the kernel over a range of
// tiles (the method is described in tdi_comb.cuh).
#include "tdi_comb.cuh"

namespace lisa {

__global__ void __launch_bounds__(kTile, 4) tdi_comb_kernel(TdiArgs a, int64_t tile_end, int G)
{
    __shared__ CombSmem s;
    const int64_t t0 = a.tile0 + (int64_t)blockIdx.x * G;
    const int nt = (int)(tile_end - t0 < G ? tile_end - t0 : G);
    comb_group(a, t0, nt, G, s);
}

// Launch over tiles [a.tile0, a.tile0 + tiles) (host side): groups of up to
// 8 tiles, never wider than one orbit-table segment, and narrower when that
// leaves fewer than 4 CTAs per SM (the tiles of a group run one after the
// other).
int launch_tdi_comb(const TdiArgs& a, int64_t tiles, cudaStream_t st)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int G = a.tab.S / kTile;
    G = G > 8 ? 8 : G;
    const int64_t fill = tiles / (4 * (int64_t)sms);
    if (fill < G) G = (int)fill;
    G = G < 2 ? 2 : G;
    const int64_t grid = (tiles + G - 1) / G;
    tdi_comb_kernel<<<(unsigned)grid, kTile, 0, st>>>(a, a.tile0 + tiles, G);
    return cuda_status(cudaGetLastError(), "tdi_comb_kernel launch");
}

}  // namespace lisa
