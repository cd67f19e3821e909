// Learned corrector of the LFA links (an addition to the paper's method: the
// paper has no learned component).
//
// The LFA link z_l at its own reception time (the LFA link formula of
// Sec. III applied to each of the six links) differs from the full link y_l
// (Sec. II, positions taken at the reception time t) by
//   y_l - z_l = eps_l z_l + (1 - k.n_l)^2/24 * T_l^2 d^2 z_l/dt^2 + ...,
//   eps_l = k.(R_s(t) - R_s(t - T_l)) / (c T_l (1 - k.n_l)) ~ k.v_s / (c (1 - k.n_l)):
// the full formula's delta_s - delta_r equals T_l (1 - k.n_l) only up to the
// sender's motion over T_l, a frequency-independent O(v/c) term that is
// applied analytically (base link z_l (1 + eps_l), v_s from the derivative of
// the orbit polynomial).  A multilayer perceptron 47 -> 64 -> 64 -> 64 -> 6
// (GELU, tanh form) predicts the rest at each output sample from:
//   [ 0,30) the 5-point stencils of z_l re-based as q_k = Tbar^k d^k z/dt^k
//           (k = 0..4; feature k*6 + l), each order divided by
//           M_k = max_l |q_k,l|;
//   [30,34) log10(M_{k+1}/M_k) / 4, clamped to [-2, 2] (a local frequency);
//   [34,40) (T_l/Tbar - 1) * 100 (arm flexing);
//   [40,46) 1 - k.n_l;
//   46      dt / Tbar (the stencils' distortion depends on omega dt as well);
// with Tbar = L/c.  Inputs and outputs are O(1) in BF16: the network output is
// scaled by s = M_2 / 8, so that the corrected link is
// z_l (1 + eps_l) + s * MLP_l.  The full TDI combine then runs on the
// corrected links.
//
// Band and checks.  The local frequency f = sqrt(M_2/M_0) / (2 pi Tbar) (exact
// for a sinusoid) selects, per sample: below the trained band the plain LFA
// link (no correction: the LFA is already closer than at the band's lower
// edge); above it the full link (the whole 256-sample tile is recomputed by
// the full links kernel).  Every spot_every-th tile, counted from the call's
// first tile inside the h grid (so every call checks one), is also recomputed with
// full links and compared (band flags and spot checks only where the retarded
// times stay on the h grid; samples whose retarded times leave it, at the grid
// ends, take the full links, the form whose boundary convention the reference
// results follow); if any compared tile differs by more than
// spot_tol (max abs difference / max abs full link over the tile), every
// remaining tile is recomputed with full links in the same call (device-side
// decision, no host synchronisation) and the failure is counted.
//
// Kernels (BF16 operands, FP32 accumulation):
//   corr_features_kernel  features, scale, band flags, optional targets
//   corr_mlp_tc_kernel    inference on the fifth-generation tensor cores
//                         (tcgen05.mma, accumulators in tensor memory), all
//                         layers fused; either on given features or fused with
//                         the features and the y = z (1 + eps) + s * MLP
//                         epilogue
//   mlp_train_tc_kernel   training: forward + MSE + backward fused on the
//                         same tensor cores; weight gradients as MMAs over the
//                         rows, accumulated in tensor memory; one partial
//                         gradient per CTA
//   grad_reduce_kernel    the partials summed in a fixed order
//   adam_kernel           Adam on FP32 master weights (summing the partials
//                         itself in training), then publishing
//   publish_kernel        FP32 biases and the BF16 weight images of both
//                         tensor-core kernels
//   corr_fallback_kernel  full links on flagged / spot / failed tiles
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>

#include "async_copy.cuh"
#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "links_tile.cuh"
#include "tcgen05.cuh"
#include "tile_geo.cuh"

namespace lisa {

constexpr int kIn = 47, kInP = 48, kWid = 64, kOut = 6, kOutP = 16;
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + kWid * kIn, kOffW2 = kOffB1 + kWid, kOffB2 = kOffW2 + kWid * kWid,
                  kOffW3 = kOffB2 + kWid, kOffB3 = kOffW3 + kWid * kWid, kOffW4 = kOffB3 + kWid,
                  kOffB4 = kOffW4 + kOut * kWid, kNParams = kOffB4 + kOut;

struct CorrStats {
    unsigned spot_tiles, spot_failed, band_tiles, fallback_tiles, call_failed, max_err_bits;
};

// GELU, tanh form, with the hardware tanh approximation (|rel err| ~ 2^-11,
// below BF16 resolution).
__device__ __forceinline__ float tanh_fast(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_f(float x)
{
    const float c = 0.7978845608028654f;
    return 0.5f * x * (1.f + tanh_fast(c * fmaf(0.044715f * x, x * x, x)));
}
// Twice the GELU, 2 GELU(x) = x (1 + tanh(x (c + c 0.044715 x^2))): five
// operations.  The inference image carries the missing 1/2 in the next
// layer's weights (a power-of-two scale, exact in BF16).
__device__ __forceinline__ float gelu2_f(float x)
{
    const float c = 0.7978845608028654f;
    const float p = fmaf(x * x, c * 0.044715f, c);
    return fmaf(x, tanh_fast(x * p), x);
}
// gelu2_f of a pair, the polynomial in packed FP32 pair instructions (one
// issue slot for both values, each lane rounded as the scalar operation).
__device__ __forceinline__ float2 gelu2_f2(float2 x)
{
    const float c = 0.7978845608028654f;
    const float2 p = __ffma2_rn(__fmul2_rn(x, x), make_float2(c * 0.044715f, c * 0.044715f), make_float2(c, c));
    const float2 xp = __fmul2_rn(x, p);
    return __ffma2_rn(x, make_float2(tanh_fast(xp.x), tanh_fast(xp.y)), x);
}
__device__ __forceinline__ float gelu_grad_f(float x)
{
    const float c = 0.7978845608028654f;
    const float t = tanh_fast(c * fmaf(0.044715f * x, x * x, x));
    return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * c * fmaf(3.f * 0.044715f, x * x, 1.f);
}

// SplitMix64 (Steele, Lea, Flood 2014): minibatch row selection.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// --------------------------------------------------------------------------
// parameters
// --------------------------------------------------------------------------
// Default initialisation: W ~ U(-1/sqrt(n_in), 1/sqrt(n_in)) from SplitMix64
// of (seed, index), biases zero.
__global__ void init_params_kernel(float* __restrict__ p, uint64_t seed)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParams) return;
    int fan_in = 0;
    if (i < kOffB1) fan_in = kIn;
    else if (i >= kOffW2 && i < kOffB2) fan_in = kWid;
    else if (i >= kOffW3 && i < kOffB3) fan_in = kWid;
    else if (i >= kOffW4 && i < kOffB4) fan_in = kWid;
    if (!fan_in) { p[i] = 0.f; return; }
    const uint64_t r = splitmix64(seed * 0x100000000ull + (uint64_t)i);
    const float u = (float)(r >> 40) * (1.f / 16777216.f);        // [0, 1)
    p[i] = (2.f * u - 1.f) * rsqrtf((float)fan_in);
}

// --------------------------------------------------------------------------
// features
// --------------------------------------------------------------------------
struct FeatArgs {
    SegTable tab;
    SkyDev sky;
    const float* z;        // [6][stride] LFA links at their own time, valid on [0, nz), zero outside
    int64_t stride, nz;
    int64_t rows;          // features for samples [0, rows)
    float r1;              // Tbar / dt
    float Tbar;
    float vfac;            // d/dt of the segment coordinate over c: 2 / (S dt c)
    float inv_half;        // 2 / S
    float dtr;             // dt / Tbar (feature 46)
    float w_lo, w_hi;      // band as limits of (omega Tbar)^2 = M2/M0
    float* feats;          // [rows][kInP]
    float* scale;          // [rows]
    float* ybase;          // [6][stride] base links z (1 + eps), or null
    int* tile_flag;        // [ceil(rows / kTile)] or null: set where above the band
    int64_t safe_lo, safe_hi;  // samples whose retarded times stay on the h grid (flags only there)
    const double* y_full;  // [6][stride] full links, or null (targets)
    const double* z_ref;   // [6][stride] or null (targets; default z)
    float* target;         // [rows][kOut] or null
};

// Geometry of a block of consecutive samples inside one orbit segment, as a
// value and a slope in the segment coordinate x at the block centre xc:
// T_l (6), k.n_l (6) and k.v/c of each spacecraft (3, from the derivative of
// its position polynomial).  A block spans at most 256 samples, over which the
// orbit turns by < 1e-4 rad: the dropped curvature is below 1e-9 of T_l and
// of k.n_l, under the FP32 rounding of the polynomials themselves.
struct CorrGeo {
    float xc;
    float v[15], s[15];
};

// Quantity q of CorrGeo at xc from the FP32 segment coefficients cfs (one
// thread per quantity).
__device__ __forceinline__ void corr_geo_one(const FeatArgs& a, const float (*cfs)[7], float xc, int q, CorrGeo& g)
{
    // p(x), p'(x), p''(x) of row `row` at xc (Horner)
    auto ev3 = [&](int row, float& p, float& d, float& dd) {
        const float* b = cfs[row];
        p = b[6];
        d = 0.f;
        dd = 0.f;
#pragma unroll
        for (int k = 5; k >= 0; --k) {
            dd = fmaf(dd, xc, d);
            d = fmaf(d, xc, p);
            p = fmaf(p, xc, b[k]);
        }
        dd *= 2.f;
    };
    const float k3[3] = {a.sky.kf[0], a.sky.kf[1], a.sky.kf[2]};
    float val = 0.f, slope = 0.f, p, d, dd;
    if (q < 6) {
        ev3(kQT + q, p, d, dd);
        val = p;
        slope = d;
    } else if (q < 12) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ev3(kQN + 3 * (q - 6) + c, p, d, dd);
            val = fmaf(k3[c], p, val);
            slope = fmaf(k3[c], d, slope);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ev3(kQR + 3 * (q - 12) + c, p, d, dd);
            val = fmaf(k3[c], d, val);
            slope = fmaf(k3[c], dd, slope);
        }
        val *= a.vfac;
        slope *= a.vfac;
    }
    g.v[q] = val;
    g.s[q] = slope;
    if (q == 0) g.xc = xc;
}

// The 5-point windows z_l(i - 2 .. i + 2) of the six links for the 32
// consecutive rows of a warp (row i in lane i % 32, every lane calls it):
// each lane loads z_l(i), the two lanes at each end one more value, and the
// rest comes from the neighbours by shuffles.  Zero off [0, nz).
__device__ __forceinline__ void corr_zwin(const FeatArgs& a, int64_t i, float (&v)[6][5])
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool edge = lane < 2 || lane >= 30;
    const int64_t ke = lane < 2 ? i - 2 : i + 2;
#pragma unroll
    for (int l = 0; l < 6; ++l) {
        const float* __restrict__ zl = a.z + (int64_t)l * a.stride;
        const float c = (i >= 0 && i < a.nz) ? zl[i] : 0.f;
        const float x = (edge && ke >= 0 && ke < a.nz) ? zl[ke] : 0.f;
        const float m2 = __shfl_sync(full, c, (lane + 30) & 31);
        const float m1 = __shfl_sync(full, c, (lane + 31) & 31);
        const float p1 = __shfl_sync(full, c, (lane + 1) & 31);
        const float p2 = __shfl_sync(full, c, (lane + 2) & 31);
        const float x1 = __shfl_sync(full, x, 1);     // z(i_1 - 2) = z(i_0 - 1)
        const float x30 = __shfl_sync(full, x, 30);   // z(i_30 + 2) = z(i_31 + 1)
        v[l][0] = lane < 2 ? x : m2;
        v[l][1] = lane == 0 ? x1 : m1;
        v[l][2] = c;
        v[l][3] = lane == 31 ? x30 : p1;
        v[l][4] = lane >= 30 ? x : p2;
    }
}

// Features of sample i (segment coordinate x) from its link windows v
// (corr_zwin) and the block geometry g: the feature row ft (ft[46] = dt/Tbar,
// ft[47] = 0), the scale s (0 below the band), eps_l, the link values z_l(i),
// and whether the local frequency is above the band.
__device__ __forceinline__ void corr_feature_row(const FeatArgs& a, const float (&v)[6][5], const CorrGeo& g,
                                                 float x, float (&ft)[kInP], float& sc, float (&eps)[6],
                                                 float (&z0)[6], bool& above)
{
    const float r1 = a.r1, r2 = r1 * r1;
    float q[5][6];
#pragma unroll
    for (int l = 0; l < 6; ++l) {
        // differences first: the stencils of slowly varying series cancel less
        const float d0 = v[l][1] - v[l][0], d1 = v[l][2] - v[l][1], d2 = v[l][3] - v[l][2], d3 = v[l][4] - v[l][3];
        q[0][l] = v[l][2];
        q[1][l] = r1 * (8.f * (d1 + d2) - (d0 + d1 + d2 + d3)) * (1.f / 12.f);
        q[2][l] = r2 * (14.f * (d2 - d1) - (d1 - d0) - (d3 - d2)) * (1.f / 12.f);
        q[3][l] = r2 * r1 * ((d0 + d1 + d2 + d3) - 2.f * (d1 + d2)) * 0.5f;
        q[4][l] = r2 * r2 * ((d3 - d2) - 2.f * (d2 - d1) + (d1 - d0));
        z0[l] = v[l][2];
    }
    float mk[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float mx = 0.f;
#pragma unroll
        for (int l = 0; l < 6; ++l) mx = fmaxf(mx, fabsf(q[k][l]));
        mk[k] = mx;
        const float inv = mx > 0.f ? 1.f / mx : 0.f;
#pragma unroll
        for (int l = 0; l < 6; ++l) ft[k * 6 + l] = q[k][l] * inv;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float lr = (mk[k] > 0.f && mk[k + 1] > 0.f) ? log10f(__fdividef(mk[k + 1], mk[k])) : -8.f;
        ft[30 + k] = fminf(fmaxf(lr, -8.f), 8.f) * 0.25f;
    }
    // geometry: linear in x about the block centre
    const float dx = x - g.xc;
    float kv[3];
#pragma unroll
    for (int s3 = 0; s3 < 3; ++s3) kv[s3] = fmaf(g.s[12 + s3], dx, g.v[12 + s3]);
#pragma unroll
    for (int l = 0; l < 6; ++l) {
        ft[34 + l] = (fmaf(g.s[l], dx, g.v[l]) / a.Tbar - 1.f) * 100.f;
        const float om = 1.f - fmaf(g.s[6 + l], dx, g.v[6 + l]);
        ft[40 + l] = om;
        eps[l] = om > 1e-6f ? __fdividef(kv[link_sender(l)], om) : 0.f;
    }
    ft[46] = a.dtr;
    ft[47] = 0.f;
    // band: (omega Tbar)^2 ~ M2/M0
    sc = 0.125f * mk[2];
    const float w2 = mk[0] > 0.f ? mk[2] / mk[0] : 0.f;
    if (!(w2 >= a.w_lo)) sc = 0.f;                    // below the band (or no signal): plain LFA link
    above = w2 > a.w_hi;
}

// FP32 copy of the coefficients of orbit segment s (every thread of the
// block calls it; no barrier inside).
__device__ __forceinline__ void load_segment_f32(const SegTable& tab, int64_t s, float (*cfs)[7])
{
    for (int e = threadIdx.x; e < kNQ * 7; e += blockDim.x)
        cfs[e / 7][e % 7] = (float)tab.coef[(s * kNQ + e / 7) * kNC + e % 7];
}

__global__ void __launch_bounds__(256) corr_features_kernel(FeatArgs a)
{
    // The block's 256 samples lie in one orbit segment (segments are whole
    // multiples of 512 samples): its coefficients are converted to FP32 once
    // (conversions from FP64 run on the FP64 pipe).
    __shared__ float cfs[kNQ][7];
    __shared__ CorrGeo geo[2];
    const int64_t b0 = (int64_t)blockIdx.x * blockDim.x;
    int64_t s = b0 / a.tab.S;
    if (s >= a.tab.nseg) s = a.tab.nseg - 1;
    load_segment_f32(a.tab, s, cfs);
    __syncthreads();
    // geometry of the block's two 128-row halves about their centres, as the
    // tensor-core kernel takes it for its 128-row tiles (same arithmetic, so
    // both give the same features and base links)
    const int t = threadIdx.x, half = t >> 7;
    if (t % 128 < 15) {
        const float xh = (float)(int)(b0 + 128 * half - s * a.tab.S) * a.inv_half - 1.f;
        corr_geo_one(a, cfs, xh + 63.5f * a.inv_half, t % 128, geo[half]);
    }
    const int64_t i = b0 + t;
    float v[6][5];
    corr_zwin(a, i, v);   // every lane of the warp
    __syncthreads();
    if (i >= a.rows) return;
    float ft[kInP], sc, eps[6], z0[6];
    bool above;
    const float x0 = (float)(int)(b0 + 128 * half - s * a.tab.S) * a.inv_half - 1.f;
    corr_feature_row(a, v, geo[half], x0 + (float)(t & 127) * a.inv_half, ft, sc, eps, z0, above);
    float4* fo = reinterpret_cast<float4*>(a.feats + i * kInP);
#pragma unroll
    for (int c = 0; c < kInP / 4; ++c) fo[c] = make_float4(ft[4 * c], ft[4 * c + 1], ft[4 * c + 2], ft[4 * c + 3]);
    if (above && a.tile_flag && i >= a.safe_lo && i < a.safe_hi) atomicOr(&a.tile_flag[i / kTile], 1);
    a.scale[i] = sc;
    if (a.ybase) {
#pragma unroll
        for (int l = 0; l < 6; ++l) a.ybase[(int64_t)l * a.stride + i] = fmaf(eps[l], z0[l], z0[l]);
    }
    if (a.target) {
#pragma unroll
        for (int l = 0; l < 6; ++l) {
            float t = 0.f;
            if (sc > 0.f && a.y_full) {
                const int64_t zi = (int64_t)l * a.stride + i;
                const double zr = a.z_ref ? a.z_ref[zi] : (double)z0[l];
                t = (float)((a.y_full[zi] - zr * (1.0 + (double)eps[l])) / (double)sc);
            }
            a.target[i * kOut + l] = t;
        }
    }
}

// --------------------------------------------------------------------------
// inference on the fifth-generation tensor cores
// --------------------------------------------------------------------------
// One CTA of four warps per 128-row tile at a time (persistent over tiles):
// thread r owns row r, which is also tensor-memory lane r of the accumulator.
// Per layer: the BF16 operand rows are written to shared memory in the
// K-major core-matrix layout, one thread issues the K/16 MMAs (128 x N x 16,
// BF16 -> FP32 in tensor memory) and commits them to an mbarrier, and each
// thread reads its accumulator row back (tcgen05.ld) for bias, GELU and the
// next operand.  Weights: a BF16 image in the same layout, fetched once per
// CTA with a bulk copy.
//
// Operand layout (bytes): element (r, k) of a K-major matrix with K/8 core
// columns sits at (r/8) * SBO + (k/8) * 128 + (r%8) * 16 + (k%8) * 2, with
// SBO = (K/8) * 128.
constexpr int kTcRows = 128;
constexpr uint32_t kTcW1 = 0, kTcW2 = 6144, kTcW3 = 14336, kTcW4 = 22528, kTcWBytes = 24576;
constexpr uint32_t kTcActSbo = 1024;   // activation tile: 8 core columns (K up to 64)

__host__ __device__ constexpr uint32_t tc_off(int r, int k, uint32_t sbo)
{
    return (uint32_t)(r >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(r & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

struct __align__(128) TcSmem {
    unsigned char w[kTcWBytes];      // weights image
    unsigned char act[16384];        // operand tile: 128 rows x 64 BF16
    float bias[3 * kWid + kOutP];
    float cfs[kNQ][7];               // FP32 orbit segment (fused mode)
    CorrGeo geo;                     // the tile's geometry (fused mode)
    int64_t cseg;
    uint64_t bar_w, bar_mma;
    uint32_t tmem_base;
};

struct TcArgs {
    const unsigned char* wimg;       // 16-byte aligned
    const float* bias;               // b1 | b2 | b3 | b4 (padded: 64, 64, 64, 16)
    int64_t rows;
    // raw mode: x [rows][kInP] -> out [rows][kOut]
    const float* x;
    float* out;
    // fused mode (x == null): features from FeatArgs, corrected links into y [6][stride]
    FeatArgs fa;
    float* y;
    unsigned int* status;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Row r of the operand tile from 8 consecutive values per 16-byte store.
__device__ __forceinline__ void store_row_bf16(unsigned char* act, int r, int kb, const float* v8)
{
    uint4 u;
    u.x = pack_bf16x2(v8[0], v8[1]);
    u.y = pack_bf16x2(v8[2], v8[3]);
    u.z = pack_bf16x2(v8[4], v8[5]);
    u.w = pack_bf16x2(v8[6], v8[7]);
    *reinterpret_cast<uint4*>(act + tc_off(r, 8 * kb, kTcActSbo)) = u;
}

// One layer: MMAs issued by thread 0 after the operand tile is complete, then
// a bounded wait for their completion.  The result is the same in every
// thread; on false the phase is left at the one that did not complete.
__device__ __forceinline__ bool tc_layer(TcSmem& sm, uint32_t wofs, uint32_t wsbo, int K, int N, uint32_t& phase)
{
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after_sync();
        const uint32_t idesc = idesc_bf16_f32(kTcRows, N);
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = smem_desc(sm.act + 2 * s * 128, 128u, kTcActSbo);
            const uint64_t bd = smem_desc(sm.w + wofs + 2 * s * 128, 128u, wsbo);
            tc_mma_bf16(sm.tmem_base, ad, bd, idesc, s > 0 ? 1u : 0u);
        }
        tc_commit(&sm.bar_mma);
    }
    const bool ok = mbar_wait_bounded(&sm.bar_mma, phase);
    const bool all_ok = __syncthreads_or(ok ? 0 : 1) == 0;
    if (all_ok) phase ^= 1u;
    tc_fence_after_sync();
    return all_ok;
}

#ifndef LISA_CORR_CTAS
#define LISA_CORR_CTAS 5
#endif
// CTAs per SM of the tensor-core kernel: shared memory allows 5, which caps
// registers at 96 per thread (a few bytes spill; measured 0.81 ms against
// 0.83 ms with 4 CTAs of 128 registers on one year at 5 s)
constexpr int kCorrCtas = LISA_CORR_CTAS;

__global__ void __launch_bounds__(kTcRows, kCorrCtas) corr_mlp_tc_kernel(TcArgs A)
{
    __shared__ TcSmem sm;
    const int t = threadIdx.x, warp = t >> 5;
    if (t == 0) {
        mbar_init(&sm.bar_w, 1);
        mbar_init(&sm.bar_mma, 1);
        mbar_init_fence();
        sm.cseg = -1;
    }
    if (warp == 0) tmem_alloc(&sm.tmem_base, 64);
    for (int e = t; e < 3 * kWid + kOutP; e += blockDim.x) sm.bias[e] = A.bias[e];
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    if (t == 0) {
        mbar_arrive_expect_tx(&sm.bar_w, kTcWBytes);
        bulk_copy_g2s(sm.w, A.wimg, kTcWBytes, &sm.bar_w);
    }
    const bool okw = __syncthreads_or(mbar_wait_bounded(&sm.bar_w, 0) ? 0 : 1) == 0;
    bool ok = okw;
    uint32_t phase = 0;
    const uint32_t lane_base = sm.tmem_base + ((uint32_t)(warp * 32) << 16);
    const int64_t ntiles = (A.rows + kTcRows - 1) / kTcRows;
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * kTcRows + t;
        const bool live = i < A.rows;
        // ---- layer-1 operand: the feature row of sample i
        float ft[kInP];
        float sc = 0.f, base[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (A.x) {
            if (live) {
                const float4* xr = reinterpret_cast<const float4*>(A.x + i * kInP);
#pragma unroll
                for (int c = 0; c < kInP / 4; ++c) {
                    const float4 v = xr[c];
                    ft[4 * c] = v.x; ft[4 * c + 1] = v.y; ft[4 * c + 2] = v.z; ft[4 * c + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < kInP; ++c) ft[c] = 0.f;
            }
        } else {
            // the tile's 128 samples lie in one orbit segment
            int64_t s = (tile * kTcRows) / A.fa.tab.S;
            if (s >= A.fa.tab.nseg) s = A.fa.tab.nseg - 1;
            if (s != sm.cseg) {
                __syncthreads();
                load_segment_f32(A.fa.tab, s, sm.cfs);
                __syncthreads();
                if (t == 0) sm.cseg = s;
            }
            // the tile's geometry about its centre row (the previous tile's
            // readers are past the layer barriers)
            const float x0 = (float)(int)(tile * kTcRows - s * A.fa.tab.S) * A.fa.inv_half - 1.f;
            if (t < 15) corr_geo_one(A.fa, sm.cfs, x0 + 63.5f * A.fa.inv_half, t, sm.geo);
            float v[6][5];
            corr_zwin(A.fa, i, v);   // every lane of the warp
            __syncthreads();
            if (live) {
                float eps[6], z0[6];
                bool above;
                corr_feature_row(A.fa, v, sm.geo, x0 + (float)t * A.fa.inv_half, ft, sc, eps, z0, above);
                if (above && A.fa.tile_flag && i >= A.fa.safe_lo && i < A.fa.safe_hi)
                    atomicOr(&A.fa.tile_flag[i / kTile], 1);
#pragma unroll
                for (int l = 0; l < 6; ++l) base[l] = fmaf(eps[l], z0[l], z0[l]);
            } else {
#pragma unroll
                for (int c = 0; c < kInP; ++c) ft[c] = 0.f;
            }
        }
#pragma unroll
        for (int kb = 0; kb < kInP / 8; ++kb) store_row_bf16(sm.act, t, kb, ft + 8 * kb);
        // ---- hidden layers
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            ok = tc_layer(sm, l == 0 ? kTcW1 : l == 1 ? kTcW2 : kTcW3, l == 0 ? 768u : 1024u, l == 0 ? kInP : kWid,
                          kWid, phase);
            if (!ok) break;
#pragma unroll
            for (int cb = 0; cb < kWid / 16; ++cb) {
                float v[16];
                tmem_ld16(lane_base + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const float2 b = *reinterpret_cast<const float2*>(&sm.bias[l * kWid + cb * 16 + k]);
                    const float2 g = gelu2_f2(__fadd2_rn(make_float2(v[k], v[k + 1]), b));
                    v[k] = g.x;
                    v[k + 1] = g.y;
                }
                store_row_bf16(sm.act, t, 2 * cb, v);
                store_row_bf16(sm.act, t, 2 * cb + 1, v + 8);
            }
        }
        if (!ok) break;
        // ---- output layer
        ok = tc_layer(sm, kTcW4, 1024u, kWid, kOutP, phase);
        if (!ok) break;
        float v[16];
        tmem_ld16(lane_base, v);
        tmem_wait_ld();
        if (live) {
            if (A.x) {
#pragma unroll
                for (int l = 0; l < kOut; ++l) A.out[i * kOut + l] = v[l] + sm.bias[3 * kWid + l];
            } else {
#pragma unroll
                for (int l = 0; l < kOut; ++l)
                    A.y[(int64_t)l * A.fa.stride + i] = fmaf(sc, v[l] + sm.bias[3 * kWid + l], base[l]);
            }
        }
    }
    if (!okw) {
        // the weights copy did not complete: flag it and give the copy another
        // bounded wait before the block leaves
        if (t == 0) flag_timeout(A.status);
        mbar_wait_bounded(&sm.bar_w, 0);
    } else if (!ok) {
        // an MMA completion wait gave up: flag it, let the MMAs finish (again
        // bounded) before releasing tensor memory
        if (t == 0) flag_timeout(A.status);
        mbar_wait_bounded(&sm.bar_mma, phase);
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(sm.tmem_base, 64);
    }
}

// --------------------------------------------------------------------------
// training on the fifth-generation tensor cores
// --------------------------------------------------------------------------
// One CTA of four warps per 128-row tile at a time (persistent over the tiles
// of the pass): thread r owns row r, which is tensor-memory lane r.
//  Forward: as in inference (plain GELU, unscaled weights), the
//    pre-activations z1..z3 kept in tensor memory for the backward pass.
//  Backward, per row: dZ4 = 2 (yhat - target) / M on the six outputs;
//    dA_l = dZ_{l+1} W_{l+1} (an MMA with the BF16 rows of dZ_{l+1} as A and
//    the image of W_{l+1}^T as B), dZ_l = dA_l * GELU'(z_l).
//  Weight gradients G_l = dZ_l^T A_{l-1} reduce over the rows: MMAs whose K
//    dimension is the tile's 128 rows, with operands stored transposed (row
//    = feature, K-major along the rows), accumulated in tensor memory over the
//    CTA's tiles.  Their M dimension (a layer's inputs, 64) is filled to 128
//    by pairing two layers in one MMA: rows (l', k) hold A_{l'-1}^T, columns
//    (l, n) hold dZ_l^T, and only the diagonal blocks l' = l are read back
//    (layers 2 and 3: one 128 x 128 accumulator; layers 1 and 4: 128 x 80).
//  Bias gradients: row sums of the transposed dZ tiles.
// Each CTA writes its partial gradient and loss; a second kernel adds the
// partials in a fixed order (run-to-run identical).
constexpr int kTrRows = 128;
// Training weight image (bytes, K-major operand layout): W_l [n][k] for the
// forward MMAs, W_l^T [k][n] for the input-gradient MMAs.
constexpr uint32_t kTrW1 = 0, kTrW2 = 6144, kTrW3 = 14336, kTrW4 = 22528;      // SBO 768, 1024, 1024, 1024
constexpr uint32_t kTrW2t = 24576, kTrW3t = 32768, kTrW4t = 40960;             // SBO 1024, 1024, 256
constexpr uint32_t kTrWBytes = 43008;
constexpr uint32_t kTrSboT = 2048;   // transposed tiles: 16 core columns (K = 128 rows)
// tensor-memory columns: paired weight-gradient accumulators, output, dA, z1..z3
constexpr uint32_t kTmD2 = 0, kTmD1 = 128, kTmOut = 224, kTmDA = 256, kTmZ1 = 320, kTmCols = 512;

struct __align__(128) TrainSmem {
    unsigned char w[kTrWBytes];
    unsigned char act[16384];     // [128 rows][64] K-major (SBO 1024): forward operand
    unsigned char dz[16384];      // [128 rows][64] K-major: backward operand
    unsigned char p1a[32768];     // [128][128 rows]: A0^T (features, rows 0..46) | A3^T
    unsigned char p1b[20480];     // [80][128 rows]:  dZ1^T | dZ4^T (rows 64..69)
    unsigned char p2a[32768];     // A1^T | A2^T
    unsigned char p2b[32768];     // dZ2^T | dZ3^T
    float bias[3 * kWid + kOutP];
    float gb[3 * kWid + kOutP];   // bias gradients of this CTA
    float loss;
    uint64_t bar_w, bar_mma;
    uint32_t tmem_base;
};
constexpr size_t kTrSmem = sizeof(TrainSmem);
static_assert(kTrSmem <= 227 * 1024, "training tile exceeds shared memory");

struct TrainArgs {
    const unsigned char* wimg;    // training image (16-byte aligned)
    const float* bias;            // b1 | b2 | b3 | b4 (padded 64, 64, 64, 16)
    const float* x;               // [n_data][kInP]
    const float* tgt;             // [n_data][kOut]
    int64_t n_data;
    int64_t M;                    // rows of this pass (batch size, or n_data)
    int sampled;                  // 1: row r is data row splitmix64(seed + r) % n_data
    uint64_t seed;
    float* part;                  // [gridDim.x][kNParams + 1]: partial gradient, then partial loss
    unsigned int* status;
};

__device__ __forceinline__ int64_t data_row(const TrainArgs& A, int64_t r)
{
    return A.sampled ? (int64_t)(splitmix64(A.seed + (uint64_t)r) % (uint64_t)A.n_data) : r;
}

// Element (row, m) of a transposed [rows][128] tile.
__device__ __forceinline__ void store_t(unsigned char* P, int row, int m, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(P + tc_off(row, m, kTrSboT)) = __float2bfloat16(v);
}

// D (+)= A . B^T over K (a multiple of 16): A rows in a K-major tile at a
// (SBO sa), B rows at b (SBO sb).  Issued by one thread.
__device__ __forceinline__ void tr_mma(uint32_t d, const unsigned char* a, uint32_t sa, const unsigned char* b,
                                       uint32_t sb, int M, int N, int K, bool acc)
{
    const uint32_t idesc = idesc_bf16_f32(M, N);
    for (int s = 0; s < K / 16; ++s)
        tc_mma_bf16(d, smem_desc(a + 256 * s, 128u, sa), smem_desc(b + 256 * s, 128u, sb), idesc,
                    (acc || s > 0) ? 1u : 0u);
}

// Operand tiles complete -> thread 0 issues `issue` -> bounded wait for the
// MMAs.  Same result in every thread; on false the phase is left at the one
// that did not complete.
template <class F>
__device__ __forceinline__ bool tr_step(TrainSmem& sm, uint32_t& phase, F issue)
{
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after_sync();
        issue();
        tc_commit(&sm.bar_mma);
    }
    const bool ok = mbar_wait_bounded(&sm.bar_mma, phase);
    const bool all_ok = __syncthreads_or(ok ? 0 : 1) == 0;
    if (all_ok) phase ^= 1u;
    tc_fence_after_sync();
    return all_ok;
}

// Sum over the 128 rows (K) of row `row` of a transposed tile.
__device__ __forceinline__ float row_sum_t(const unsigned char* P, int row)
{
    float s = 0.f;
#pragma unroll 4
    for (int cb = 0; cb < kTrRows / 8; ++cb) {
        const uint4 u = *reinterpret_cast<const uint4*>(P + tc_off(row, 8 * cb, kTrSboT));
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(h[q]);
            s += f.x + f.y;
        }
    }
    return s;
}

__global__ void __launch_bounds__(kTrRows, 1) mlp_train_tc_kernel(TrainArgs A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;
    if (t == 0) {
        mbar_init(&sm.bar_w, 1);
        mbar_init(&sm.bar_mma, 1);
        mbar_init_fence();
        sm.loss = 0.f;
    }
    if (warp == 0) tmem_alloc(&sm.tmem_base, kTmCols);
    for (int e = t; e < 3 * kWid + kOutP; e += blockDim.x) {
        sm.bias[e] = A.bias[e];
        sm.gb[e] = 0.f;
    }
    // transposed tiles start at zero (their padding rows are never written)
    {
        uint4* z = reinterpret_cast<uint4*>(sm.p1a);
        const int n16 = (32768 + 20480 + 32768 + 32768) / 16;
        for (int e = t; e < n16; e += blockDim.x) z[e] = make_uint4(0u, 0u, 0u, 0u);
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    if (t == 0) {
        mbar_arrive_expect_tx(&sm.bar_w, kTrWBytes);
        bulk_copy_g2s(sm.w, A.wimg, kTrWBytes, &sm.bar_w);
    }
    const bool okw = __syncthreads_or(mbar_wait_bounded(&sm.bar_w, 0) ? 0 : 1) == 0;
    bool ok = okw;
    uint32_t phase = 0;
    const uint32_t tb = sm.tmem_base;
    const uint32_t lane = tb + ((uint32_t)(warp * 32) << 16);
    const float inv_m = 1.f / (float)A.M;
    const int64_t ntiles = (A.M + kTrRows - 1) / kTrRows;
    bool first = true;
    float lsum = 0.f;
    const uint32_t wf[4] = {kTrW1, kTrW2, kTrW3, kTrW4};
    const uint32_t wt[4] = {0u, kTrW2t, kTrW3t, kTrW4t};
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int64_t r = tile * kTrRows + t;
        const bool live = r < A.M;
        const int64_t dr = live ? data_row(A, r) : 0;
        // ---- layer-1 operand, its transposed copy, and the target row
        float ft[kInP];
        if (live) {
            const float4* xr = reinterpret_cast<const float4*>(A.x + dr * kInP);
#pragma unroll
            for (int c = 0; c < kInP / 4; ++c) {
                const float4 v = xr[c];
                ft[4 * c] = v.x; ft[4 * c + 1] = v.y; ft[4 * c + 2] = v.z; ft[4 * c + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int c = 0; c < kInP; ++c) ft[c] = 0.f;
        }
        ft[kIn] = 0.f;
#pragma unroll
        for (int kb = 0; kb < kInP / 8; ++kb) store_row_bf16(sm.act, t, kb, ft + 8 * kb);
#pragma unroll
        for (int k = 0; k < kIn; ++k) store_t(sm.p1a, k, t, ft[k]);
        float tg[kOut];
#pragma unroll
        for (int l = 0; l < kOut; ++l) tg[l] = live ? A.tgt[dr * kOut + l] : 0.f;
        // ---- forward: hidden layers (a1 -> p2a rows 0.., a2 -> p2a rows 64.., a3 -> p1a rows 64..)
#pragma unroll 1
        for (int l = 0; l < 3; ++l) {
            const uint32_t zc = kTmZ1 + 64u * (uint32_t)l;
            ok = tr_step(sm, phase, [&] {
                tr_mma(tb + zc, sm.act, 1024u, sm.w + wf[l], l == 0 ? 768u : 1024u, kTrRows, kWid,
                       l == 0 ? kInP : kWid, false);
            });
            if (!ok) break;
            unsigned char* P = l == 2 ? sm.p1a : sm.p2a;
            const int roff = l == 0 ? 0 : 64;
#pragma unroll
            for (int cb = 0; cb < kWid / 16; ++cb) {
                float v[16];
                tmem_ld16(lane + zc + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = live ? gelu_f(v[k] + sm.bias[l * kWid + cb * 16 + k]) : 0.f;
                store_row_bf16(sm.act, t, 2 * cb, v);
                store_row_bf16(sm.act, t, 2 * cb + 1, v + 8);
#pragma unroll
                for (int k = 0; k < 16; ++k) store_t(P, roff + cb * 16 + k, t, v[k]);
            }
        }
        if (!ok) break;
        // ---- output layer, loss and dZ4 (-> dz, p1b rows 64..79)
        ok = tr_step(sm, phase, [&] { tr_mma(tb + kTmOut, sm.act, 1024u, sm.w + kTrW4, 1024u, kTrRows, kOutP, kWid, false); });
        if (!ok) break;
        {
            float v[16], d[16];
            tmem_ld16(lane + kTmOut, v);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                d[c] = 0.f;
                if (c < kOut && live) {
                    const float diff = v[c] + sm.bias[3 * kWid + c] - tg[c];
                    lsum = fmaf(diff, diff, lsum);
                    d[c] = 2.f * diff * inv_m;
                }
            }
            store_row_bf16(sm.dz, t, 0, d);
            store_row_bf16(sm.dz, t, 1, d + 8);
#pragma unroll
            for (int c = 0; c < 16; ++c) store_t(sm.p1b, 64 + c, t, d[c]);
        }
        // ---- hidden layers, top down (dZ3 -> p2b rows 64.., dZ2 -> p2b rows 0.., dZ1 -> p1b rows 0..)
#pragma unroll 1
        for (int l = 2; l >= 0; --l) {
            ok = tr_step(sm, phase, [&] {
                tr_mma(tb + kTmDA, sm.dz, 1024u, sm.w + wt[l + 1], l == 2 ? 256u : 1024u, kTrRows, kWid,
                       l == 2 ? kOutP : kWid, false);
            });
            if (!ok) break;
            const uint32_t zc = kTmZ1 + 64u * (uint32_t)l;
            unsigned char* P = l == 0 ? sm.p1b : sm.p2b;
            const int roff = l == 2 ? 64 : 0;
#pragma unroll
            for (int cb = 0; cb < kWid / 16; ++cb) {
                float da[16], z[16], d[16];
                tmem_ld16(lane + kTmDA + cb * 16, da);
                tmem_ld16(lane + zc + cb * 16, z);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    d[k] = live ? da[k] * gelu_grad_f(z[k] + sm.bias[l * kWid + cb * 16 + k]) : 0.f;
                if (l > 0) {
                    store_row_bf16(sm.dz, t, 2 * cb, d);
                    store_row_bf16(sm.dz, t, 2 * cb + 1, d + 8);
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) store_t(P, roff + cb * 16 + k, t, d[k]);
            }
        }
        if (!ok) break;
        // ---- weight gradients of the tile, accumulated over the CTA's tiles
        const bool acc = !first;
        ok = tr_step(sm, phase, [&] {
            tr_mma(tb + kTmD2, sm.p2a, kTrSboT, sm.p2b, kTrSboT, kTrRows, 128, kTrRows, acc);
            tr_mma(tb + kTmD1, sm.p1a, kTrSboT, sm.p1b, kTrSboT, kTrRows, 80, kTrRows, acc);
        });
        first = false;
        if (!ok) break;
        // bias gradients: row sums of the transposed dZ tiles (thread t owns row t)
        sm.gb[(t < 64 ? kWid : 2 * kWid) + (t & 63)] += row_sum_t(sm.p2b, t);
        if (t < 64) sm.gb[t] += row_sum_t(sm.p1b, t);
        else if (t < 64 + kOut) sm.gb[3 * kWid + t - 64] += row_sum_t(sm.p1b, t);
    }
    if (ok) {
        float* P = A.part + (int64_t)blockIdx.x * (kNParams + 1);
        const bool hi = t >= 64;
        const int k = t & 63;
        if (first) {
            for (int e = t; e < kNParams + 1; e += blockDim.x) P[e] = 0.f;
        } else {
            // layers 2 (lanes 0..63) and 3 (lanes 64..127): G_l[n][k] = D2[(l, k)][(l, n)]
#pragma unroll
            for (int cb = 0; cb < kWid / 16; ++cb) {
                float v[16];
                tmem_ld16(lane + kTmD2 + (hi ? 64u : 0u) + cb * 16, v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) P[(hi ? kOffW3 : kOffW2) + (cb * 16 + j) * kWid + k] = v[j];
            }
            // layers 1 (lanes 0..46, columns 0..63) and 4 (lanes 64..127, columns 64..69)
            if (!hi) {
#pragma unroll
                for (int cb = 0; cb < kWid / 16; ++cb) {
                    float v[16];
                    tmem_ld16(lane + kTmD1 + cb * 16, v);
                    tmem_wait_ld();
                    if (k < kIn) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) P[kOffW1 + (cb * 16 + j) * kIn + k] = v[j];
                    }
                }
            } else {
                float v[16];
                tmem_ld16(lane + kTmD1 + 64u, v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < kOut; ++j) P[kOffW4 + j * kWid + k] = v[j];
            }
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if ((t & 31) == 0) atomicAdd(&sm.loss, lsum);
            __syncthreads();
            if (t < kWid) {
                P[kOffB1 + t] = sm.gb[t];
                P[kOffB2 + t] = sm.gb[kWid + t];
                P[kOffB3 + t] = sm.gb[2 * kWid + t];
            }
            if (t < kOut) P[kOffB4 + t] = sm.gb[3 * kWid + t];
            if (t == 0) P[kNParams] = sm.loss * inv_m;
        }
    } else {
        if (t == 0) flag_timeout(A.status);
        if (!okw) mbar_wait_bounded(&sm.bar_w, 0);
        else mbar_wait_bounded(&sm.bar_mma, phase);
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(sm.tmem_base, kTmCols);
    }
}

// grad[i] = sum over the CTA partials in order (i < kNParams); loss likewise.
__global__ void grad_reduce_kernel(const float* __restrict__ part, int nblk, float* __restrict__ grad,
                                   float* __restrict__ loss)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kNParams) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * (kNParams + 1) + i];
    if (i < kNParams) grad[i] = s;
    else if (loss) *loss = s;
}

// --------------------------------------------------------------------------
// publishing the parameters: FP32 biases (padded) and the BF16 images of the
// inference kernel (W/2 after a GELU, see gelu2_f) and of the training kernel
// --------------------------------------------------------------------------
struct ParamImages {
    float* bias;            // b1 | b2 | b3 | b4 padded (64, 64, 64, 16)
    unsigned char* inf;     // inference image (kTcWBytes)
    unsigned char* train;   // training image (kTrWBytes)
};

// Write parameter i (value v) into every image that holds it.  Padding
// entries are not touched (zero since creation).
__device__ __forceinline__ void publish_param(const ParamImages& im, int64_t i, float v)
{
    __nv_bfloat16* fi = (__nv_bfloat16*)im.inf;
    __nv_bfloat16* ft = (__nv_bfloat16*)im.train;
    const __nv_bfloat16 b = __float2bfloat16(v), bh = __float2bfloat16(0.5f * v);
    if (i < kOffB1) {                       // W1 [64][47]
        const int n = (int)(i / kIn), k = (int)(i % kIn);
        fi[(kTcW1 + tc_off(n, k, 768)) / 2] = b;
        ft[(kTrW1 + tc_off(n, k, 768)) / 2] = b;
    } else if (i < kOffW2) {
        im.bias[i - kOffB1] = v;
    } else if (i < kOffB2 || (i >= kOffW3 && i < kOffB3)) {   // W2, W3 [64][64]
        const bool l3 = i >= kOffW3;
        const int64_t j = i - (l3 ? kOffW3 : kOffW2);
        const int n = (int)(j / kWid), k = (int)(j % kWid);
        fi[((l3 ? kTcW3 : kTcW2) + tc_off(n, k, 1024)) / 2] = bh;
        ft[((l3 ? kTrW3 : kTrW2) + tc_off(n, k, 1024)) / 2] = b;
        ft[((l3 ? kTrW3t : kTrW2t) + tc_off(k, n, 1024)) / 2] = b;
    } else if (i < kOffW3) {
        im.bias[kWid + i - kOffB2] = v;
    } else if (i < kOffW4) {
        im.bias[2 * kWid + i - kOffB3] = v;
    } else if (i < kOffB4) {                // W4 [6][64]
        const int64_t j = i - kOffW4;
        const int n = (int)(j / kWid), k = (int)(j % kWid);
        fi[(kTcW4 + tc_off(n, k, 1024)) / 2] = bh;
        ft[(kTrW4 + tc_off(n, k, 1024)) / 2] = b;
        ft[(kTrW4t + tc_off(k, n, 256)) / 2] = b;
    } else if (i < kNParams) {
        im.bias[3 * kWid + i - kOffB4] = v;
    }
}

__global__ void publish_kernel(const float* __restrict__ p, ParamImages im)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParams) publish_param(im, i, p[i]);
}

// Adam (Kingma & Ba 2015) with bias correction (c1 = 1 - beta1^t,
// c2 = 1 - beta2^t) on the FP32 master parameters, then publishing.  The
// gradient is g, or, if g is null, the sum of the nblk training partials.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, const float* __restrict__ part,
                            int nblk, float* __restrict__ loss, float* __restrict__ mom, float* __restrict__ vel,
                            float lr, float b1, float b2, float eps, float c1, float c2, ParamImages im)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kNParams) return;
    float gi;
    if (g) {
        if (i == kNParams) return;
        gi = g[i];
    } else {
        gi = 0.f;
        for (int b = 0; b < nblk; ++b) gi += part[(int64_t)b * (kNParams + 1) + i];
        if (i == kNParams) {
            if (loss) *loss = gi;
            return;
        }
    }
    const float mi = b1 * mom[i] + (1.f - b1) * gi;
    const float vi = b2 * vel[i] + (1.f - b2) * gi * gi;
    mom[i] = mi;
    vel[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    publish_param(im, i, pi);
}

// --------------------------------------------------------------------------
// full-link fallback and spot checks
// --------------------------------------------------------------------------
struct FallbackArgs {
    LinksArgs la;          // y = the corrected links, overwritten where recomputed
    const int* tile_flag;  // per tile: nonzero = above the band
    int spot_every;        // 0: no spot checks
    float spot_tol;
    int global_pass;       // 0: flagged and spot tiles; 1: all others if this call failed a spot check
    int64_t safe_lo, safe_hi;  // spot checks only on tiles inside [safe_lo, safe_hi)
    int64_t spot0;         // first tile inside: spot checks on spot0, spot0 + spot_every, ...
    CorrStats* stats;
};

__global__ void __launch_bounds__(kTile) corr_fallback_kernel(FallbackArgs A)
{
    __shared__ TileGeo g;
    __shared__ LinksTile<true> s;
    __shared__ float red[2][kTile / 32];
    const LinksArgs& a = A.la;
    const int64_t tile = a.tile0 + blockIdx.x;
    const int flag = A.tile_flag[tile];
    const bool inside = tile * kTile >= A.safe_lo && (tile + 1) * kTile <= A.safe_hi;
    const bool spot = A.spot_every > 0 && inside && ((tile - A.spot0) % A.spot_every) == 0;
    if (A.global_pass) {
        if (flag || spot || A.stats->call_failed == 0) return;
    } else if (!flag && !spot && inside) {
        return;
    }
    const int64_t i0 = tile * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    tile_geo_load(g, a.tab, ic, a.sky);
    links_tile_prologue<true>(a, g, ic, i0, i0 + kTile - 1, s);
    const int64_t i = i0 + threadIdx.x;
    const bool valid = i >= a.i_begin && i < a.i_end;
    float* y = (float*)a.y;
    const bool check = !A.global_pass && spot && !flag;
    float old[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid && check) {
#pragma unroll
        for (int l = 0; l < 6; ++l) old[l] = y[l * a.ny + i];
    }
    // edge tiles outside the band and the checks: full links only on the
    // samples whose retarded times leave the h grid
    const bool whole = A.global_pass || flag || spot;
    if (valid && (whole || i < A.safe_lo || i >= A.safe_hi)) links_sample<true>(a, g, ic, i, s, y + i, a.ny);
    // a spot-checked tile keeps its corrected links unless the check fails
    // (the FP32 full links are the less accurate ones at low frequency)
    if (!check) {
        if (threadIdx.x == 0 && (A.global_pass || flag))
            atomicAdd(A.global_pass ? &A.stats->fallback_tiles : &A.stats->band_tiles, 1u);
        return;
    }
    // The FP32 full link is itself uncertain by about its interpolation
    // rounding (~5e-7 of |h|) divided by 2 (1 - k.n_l): differences within
    // that bound (1e-6 |h|max / (1 - k.n_l)) are not counted.
    float hmax = 0.f;
    for (int k = threadIdx.x; k < s.wlen; k += blockDim.x) hmax = fmaxf(hmax, fmaxf(fabsf(s.win[k].x), fabsf(s.win[k].y)));
    for (int o = 16; o > 0; o >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = hmax;
    __syncthreads();
    hmax = red[0][0];
    for (int w = 1; w < kTile / 32; ++w) hmax = fmaxf(hmax, red[0][w]);
    if (s.wlen == 0) hmax = 0.f;
    __syncthreads();
    float num = 0.f, den = 0.f;
    if (valid) {
#pragma unroll
        for (int l = 0; l < 6; ++l) {
            const float kn = (float)(a.sky.k[0] * g.b[kQN + 3 * l][0] + a.sky.k[1] * g.b[kQN + 3 * l + 1][0]
                                     + a.sky.k[2] * g.b[kQN + 3 * l + 2][0]);
            const float eb = 1e-6f * hmax / fmaxf(1.f - kn, 1e-6f);
            const float v = y[l * a.ny + i];
            num = fmaxf(num, fabsf(v - old[l]) - eb);
            den = fmaxf(den, fabsf(v));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        num = fmaxf(num, __shfl_xor_sync(0xffffffffu, num, o));
        den = fmaxf(den, __shfl_xor_sync(0xffffffffu, den, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = num;
        red[1][threadIdx.x >> 5] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kTile / 32; ++w) {
            num = fmaxf(num, red[0][w]);
            den = fmaxf(den, red[1][w]);
        }
        const float rel = den > 0.f ? fmaxf(num, 0.f) / den : 0.f;
        const bool pass = rel <= A.spot_tol;
        atomicAdd(&A.stats->spot_tiles, 1u);
        atomicMax(&A.stats->max_err_bits, __float_as_uint(rel));
        if (!pass) {
            atomicAdd(&A.stats->spot_failed, 1u);
            atomicAdd(&A.stats->call_failed, 1u);
        }
        red[0][0] = pass ? 1.f : 0.f;
    }
    __syncthreads();
    if (red[0][0] != 0.f && valid) {
#pragma unroll
        for (int l = 0; l < 6; ++l) y[l * a.ny + i] = old[l];
    }
}

}  // namespace lisa

using namespace lisa;

struct lisa_corrector {
    float* p = nullptr;       // FP32 master parameters
    float* mom = nullptr;     // Adam moments
    float* vel = nullptr;
    float* bias = nullptr;    // FP32 biases, padded (64, 64, 64, 16)
    unsigned char* wimg = nullptr;    // BF16 weights, inference image (tensor-core operand layout)
    unsigned char* wtrain = nullptr;  // BF16 weights, training image
    float* part = nullptr;    // training partials: [SMs][n_params + 1]
    int part_rows = 0;
    CorrStats* stats = nullptr;
    float* grad = nullptr;    // gradient buffer of lisa_corrector_gradient callers
    int64_t step = 0;
    double f_lo = 1e-4, f_hi = 2e-2;
    int spot_every = 64;
    float spot_tol = 0.05f;
};

namespace lisa {

static ParamImages images(const lisa_corrector* c)
{
    return ParamImages{c->bias, c->wimg, c->wtrain};
}

// All parameters into the images (their padding is zero since creation).
static int publish(lisa_corrector* c, cudaStream_t st)
{
    prof_before("corr_publish", st);
    publish_kernel<<<(unsigned)((kNParams + 255) / 256), 256, 0, st>>>(c->p, images(c));
    prof_after(st);
    return cuda_status(cudaGetLastError(), "publish_kernel launch");
}

static int sm_count()
{
    static int n[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!n[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        n[dev] = v > 0 ? v : 148;
    }
    return n[dev];
}

// The tensor-core MLP over `rows` rows: raw (x -> out) or fused with the
// features (fa, y).  Persistent: up to 4 CTAs per SM.
static int run_mlp_tc(const lisa_corrector* c, int64_t rows, const float* x, float* out, const FeatArgs* fa,
                      float* y, cudaStream_t st)
{
    if (rows <= 0) return LISA_OK;
    TcArgs A;
    memset(&A, 0, sizeof(A));
    A.wimg = c->wimg;
    A.bias = c->bias;
    A.rows = rows;
    A.x = x;
    A.out = out;
    if (fa) A.fa = *fa;
    A.y = y;
    A.status = device_status_ptr();
    const int64_t tiles = (rows + kTcRows - 1) / kTcRows;
    const int64_t cap = (int64_t)sm_count() * kCorrCtas;
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    prof_before(x ? "mlp_forward_tc" : "corr_fused_tc", st);
    corr_mlp_tc_kernel<<<grid, kTcRows, 0, st>>>(A);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "corr_mlp_tc_kernel launch");
}

static void free_corrector(lisa_corrector* c)
{
    cudaFree(c->p);
    cudaFree(c->mom);
    cudaFree(c->vel);
    cudaFree(c->bias);
    cudaFree(c->wimg);
    cudaFree(c->wtrain);
    cudaFree(c->part);
    cudaFree(c->stats);
    cudaFree(c->grad);
    delete c;
}

// One pass of the tensor-core training kernel over M rows (batch > 0: rows
// drawn from the data by SplitMix64(seed + r)), partials into c->part; the
// number of partial rows written is returned in *nblk.
static int run_train_tc(lisa_corrector* c, const float* feats, const float* target, int64_t n_data, int64_t batch,
                        uint64_t seed, int* nblk, cudaStream_t st)
{
    static int attr_dev = -1;
    int dev = 0;
    LISA_TRY(cuda_status(cudaGetDevice(&dev), "cudaGetDevice"));
    if (attr_dev != dev) {
        LISA_TRY(cuda_status(cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)kTrSmem), "cudaFuncSetAttribute"));
        attr_dev = dev;
    }
    TrainArgs A;
    A.wimg = c->wtrain;
    A.bias = c->bias;
    A.x = feats;
    A.tgt = target;
    A.n_data = n_data;
    A.M = batch > 0 ? batch : n_data;
    A.sampled = batch > 0;
    A.seed = seed;
    A.part = c->part;
    A.status = device_status_ptr();
    const int64_t tiles = (A.M + kTrRows - 1) / kTrRows;
    const int grid = (int)(tiles < c->part_rows ? tiles : c->part_rows);
    prof_before("mlp_train_tc", st);
    mlp_train_tc_kernel<<<(unsigned)grid, kTrRows, kTrSmem, st>>>(A);
    prof_after(st);
    *nblk = grid;
    return cuda_status(cudaGetLastError(), "mlp_train_tc_kernel launch");
}

static int adam_launch(lisa_corrector* c, const float* grad, int nblk, float* loss, float lr, cudaStream_t st)
{
    c->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - pow(b1, (double)c->step)), c2 = (float)(1.0 - pow(b2, (double)c->step));
    prof_before("mlp_adam", st);
    adam_kernel<<<(unsigned)((kNParams + 1 + 255) / 256), 256, 0, st>>>(c->p, grad, c->part, nblk, loss, c->mom,
                                                                        c->vel, lr, (float)b1, (float)b2, 1e-8f, c1,
                                                                        c2, images(c));
    prof_after(st);
    return cuda_status(cudaGetLastError(), "adam_kernel launch");
}

static FeatArgs make_feat_args(const SegTable& tab, const SkyDev& sky, double Tbar, double dt, const float* z,
                               int64_t stride, int64_t nz, int64_t rows, double f_lo, double f_hi, float* feats,
                               float* scale, float* ybase, int* tile_flag, int64_t safe_lo, int64_t safe_hi,
                               const double* y_full, const double* z_ref, float* target)
{
    const double two_pi_T = 2.0 * M_PI * Tbar;
    FeatArgs a;
    a.tab = tab;
    a.sky = sky;
    a.z = z;
    a.stride = stride;
    a.nz = nz;
    a.rows = rows;
    a.r1 = (float)(Tbar / dt);
    a.Tbar = (float)Tbar;
    a.vfac = (float)(2.0 / ((double)tab.S * dt * kC));
    a.inv_half = (float)(2.0 / (double)tab.S);
    a.dtr = (float)(dt / Tbar);
    a.w_lo = (float)(two_pi_T * f_lo * two_pi_T * f_lo);
    a.w_hi = isfinite(f_hi) ? (float)(two_pi_T * f_hi * two_pi_T * f_hi) : INFINITY;
    a.feats = feats;
    a.scale = scale;
    a.ybase = ybase;
    a.tile_flag = tile_flag;
    a.safe_lo = safe_lo;
    a.safe_hi = safe_hi;
    a.y_full = y_full;
    a.z_ref = z_ref;
    a.target = target;
    return a;
}

static int run_features(const SegTable& tab, const SkyDev& sky, double Tbar, double dt, const float* z,
                        int64_t stride, int64_t nz, int64_t rows, double f_lo, double f_hi, float* feats,
                        float* scale, float* ybase, int* tile_flag, int64_t safe_lo, int64_t safe_hi,
                        const double* y_full, const double* z_ref, float* target, cudaStream_t st)
{
    if (rows <= 0) return LISA_OK;
    const FeatArgs a = make_feat_args(tab, sky, Tbar, dt, z, stride, nz, rows, f_lo, f_hi, feats, scale, ybase,
                                      tile_flag, safe_lo, safe_hi, y_full, z_ref, target);
    prof_before("corr_features", st);
    corr_features_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "corr_features_kernel launch");
}

// Output samples [lo, hi) whose retarded times t - k.R/c - T (|k.R/c| <= 1 AU/c)
// and their 32-point stencils stay on the h grid.  Nearer the ends both link
// forms see the zero padding of h, and neither band flags nor spot checks
// are meaningful there.
static void safe_range(const lisa_grid& out, const lisa_grid& hg, double Tmax, int64_t& lo, int64_t& hi)
{
    const double reach = kAU / kC + 2.0 * Tmax + 20.0 * hg.dt;
    const double a = (hg.t0 + reach - out.t0) / out.dt;
    const double b = (hg.t0 + (double)hg.n * hg.dt - reach - out.t0) / out.dt;
    lo = a <= 0.0 ? 0 : (a >= (double)out.n ? out.n : (int64_t)ceil(a));
    hi = b <= 0.0 ? 0 : (b >= (double)out.n ? out.n : (int64_t)floor(b));
    if (hi < lo) hi = lo;
}

// Corrected links on out-grid samples [0, rows) into y ([6][out.n], FP32):
// LFA z, features, MLP with the y = z + s*MLP epilogue, then full links on
// tiles above the band, spot checks, and the all-tile fallback pass.
static int corrected_links(lisa_corrector* c, const lisa_orbit* orbit, const lisa_sky* sky, const lisa_grid& h_grid,
                           const void* hp, const void* hc, const lisa_grid& out, const SegTable& tab,
                           int64_t rows, float* y, Scratch& sc, cudaStream_t st)
{
    const int64_t n = out.n;
    if (rows <= 0) return LISA_OK;
    const int64_t nz = rows + 2 < n ? rows + 2 : n;
    const int64_t ntile = (rows + kTile - 1) / kTile;
    float* z = (float*)sc.alloc(sizeof(float) * 6 * (size_t)n);
    int* flags = (int*)sc.alloc(sizeof(int) * (size_t)ntile);
    if (!z || !flags) return sc.status();
    const SkyDev skyd = make_sky_dev(*sky);
    BlendSpec none{};
    LISA_TRY(launch_lfa(tab, skyd, orbit->L_m, h_grid, hp, hc, LISA_MIXED, kLfaOwnTime, LISA_LFA_UNEQUAL, LISA_XYZ,
                        out, z, nullptr, 0, nz, none, st));
    LISA_TRY(cuda_status(cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)ntile, st), "cudaMemsetAsync"));
    LISA_TRY(cuda_status(cudaMemsetAsync(&c->stats->call_failed, 0, sizeof(unsigned), st), "cudaMemsetAsync"));
    const double Tbar = orbit->L_m / kC;
    int64_t safe_lo, safe_hi;
    safe_range(out, h_grid, max_light_time(orbit, out), safe_lo, safe_hi);
    // the feature stencils of the first two rows reach z before the grid's
    // start (zero): those rows take full links, and the first tile is neither
    // band-flagged nor spot-checked
    if (safe_lo < 2) safe_lo = rows < 2 ? rows : 2;
    if (safe_hi < safe_lo) safe_hi = safe_lo;
    // features, network and z (1 + eps) + s * MLP in one tensor-core kernel
    const FeatArgs fa = make_feat_args(tab, skyd, Tbar, out.dt, z, n, nz, rows, c->f_lo, c->f_hi, nullptr, nullptr,
                                       nullptr, flags, safe_lo, safe_hi, nullptr, nullptr, nullptr);
    LISA_TRY(run_mlp_tc(c, rows, nullptr, nullptr, &fa, y, st));
    FallbackArgs A;
    A.la.tab = tab;
    A.la.sky = skyd;
    A.la.hm = make_grid_map(out, h_grid);
    A.la.hp = hp;
    A.la.hc = hc;
    A.la.y = y;
    A.la.ny = n;
    A.la.i_begin = 0;
    A.la.i_end = rows;
    A.la.tile0 = 0;
    A.tile_flag = flags;
    A.spot_every = c->spot_every;
    A.spot_tol = c->spot_tol;
    A.stats = c->stats;
    A.safe_lo = safe_lo;
    A.safe_hi = safe_hi;
    A.spot0 = (safe_lo + kTile - 1) / kTile;   // every call checks its first inside tile
    for (int pass = 0; pass < 2; ++pass) {
        A.global_pass = pass;
        prof_before(pass ? "corr_fallback_all" : "corr_fallback", st);
        corr_fallback_kernel<<<(unsigned)ntile, kTile, 0, st>>>(A);
        prof_after(st);
        LISA_TRY(cuda_status(cudaGetLastError(), "corr_fallback_kernel launch"));
    }
    return LISA_OK;
}

}  // namespace lisa

extern "C" {

int64_t lisa_corrector_num_params(void) { return kNParams; }
int lisa_corrector_num_features(void) { return kIn; }

int lisa_corrector_create(lisa_corrector** out, const float* host_params, int64_t n_params, uint64_t seed)
{
    if (!out) { set_error("lisa_corrector_create: out is NULL"); return LISA_EINVAL; }
    if (host_params && n_params != kNParams) {
        set_error("lisa_corrector_create: need %lld FP32 parameters (got %lld)", (long long)kNParams,
                  (long long)n_params);
        return LISA_EINVAL;
    }
    lisa_corrector* c = new (std::nothrow) lisa_corrector();
    if (!c) { set_error("lisa_corrector_create: out of host memory"); return LISA_ENOMEM; }
    const size_t pb = sizeof(float) * kNParams;
    const size_t bb = sizeof(float) * (3 * kWid + kOutP);
    c->part_rows = sm_count();
    int rc = cuda_status(cudaMalloc(&c->p, pb), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->mom, pb), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->vel, pb), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->bias, bb), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->stats, sizeof(CorrStats)), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->grad, pb), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->wimg, kTcWBytes), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->wtrain, kTrWBytes), "cudaMalloc");
    if (!rc) rc = cuda_status(cudaMalloc(&c->part, sizeof(float) * (size_t)c->part_rows * (kNParams + 1)), "cudaMalloc");
    if (rc) { free_corrector(c); return rc; }
    // image padding stays zero: publishing writes parameter entries only
    rc = cuda_status(cudaMemset(c->bias, 0, bb), "cudaMemset");
    if (!rc) rc = cuda_status(cudaMemset(c->wimg, 0, kTcWBytes), "cudaMemset");
    if (!rc) rc = cuda_status(cudaMemset(c->wtrain, 0, kTrWBytes), "cudaMemset");
    if (rc) {
    } else if (host_params) {
        rc = cuda_status(cudaMemcpy(c->p, host_params, pb, cudaMemcpyHostToDevice), "cudaMemcpy");
    } else {
        prof_before("corr_init", 0);
        init_params_kernel<<<(unsigned)((kNParams + 255) / 256), 256>>>(c->p, seed);
        prof_after(0);
        rc = cuda_status(cudaGetLastError(), "init_params_kernel launch");
    }
    if (!rc) rc = cuda_status(cudaMemset(c->mom, 0, pb), "cudaMemset");
    if (!rc) rc = cuda_status(cudaMemset(c->vel, 0, pb), "cudaMemset");
    if (!rc) rc = cuda_status(cudaMemset(c->stats, 0, sizeof(CorrStats)), "cudaMemset");
    if (!rc) rc = publish(c, 0);
    if (!rc) rc = cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    if (rc) { free_corrector(c); return rc; }
    *out = c;
    return LISA_OK;
}

int lisa_corrector_destroy(lisa_corrector* c)
{
    if (c) free_corrector(c);
    return LISA_OK;
}

int lisa_corrector_configure(lisa_corrector* c, double f_lo, double f_hi, int spot_every, double spot_tol)
{
    if (!c || !(f_lo >= 0.0) || !(f_hi > f_lo) || spot_every < 0 || !(spot_tol > 0.0)) {
        set_error("lisa_corrector_configure: need 0 <= f_lo < f_hi, spot_every >= 0, spot_tol > 0");
        return LISA_EINVAL;
    }
    c->f_lo = f_lo;
    c->f_hi = f_hi;
    c->spot_every = spot_every;
    c->spot_tol = (float)spot_tol;
    return LISA_OK;
}

int lisa_corrector_get_state(const lisa_corrector* c, float* params, float* adam_m, float* adam_v, int64_t* step,
                             int64_t n_params)
{
    if (!c || n_params != kNParams) { set_error("lisa_corrector_get_state: bad arguments"); return LISA_EINVAL; }
    const size_t pb = sizeof(float) * kNParams;
    int rc = cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    if (!rc && params) rc = cuda_status(cudaMemcpy(params, c->p, pb, cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (!rc && adam_m) rc = cuda_status(cudaMemcpy(adam_m, c->mom, pb, cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (!rc && adam_v) rc = cuda_status(cudaMemcpy(adam_v, c->vel, pb, cudaMemcpyDeviceToHost), "cudaMemcpy");
    if (!rc && step) *step = c->step;
    return rc;
}

int lisa_corrector_set_state(lisa_corrector* c, const float* params, const float* adam_m, const float* adam_v,
                             int64_t step, int64_t n_params)
{
    if (!c || n_params != kNParams || step < 0) { set_error("lisa_corrector_set_state: bad arguments"); return LISA_EINVAL; }
    const size_t pb = sizeof(float) * kNParams;
    int rc = cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    if (!rc && params) rc = cuda_status(cudaMemcpy(c->p, params, pb, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (!rc && adam_m) rc = cuda_status(cudaMemcpy(c->mom, adam_m, pb, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (!rc && adam_v) rc = cuda_status(cudaMemcpy(c->vel, adam_v, pb, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (!rc) c->step = step;
    if (!rc) rc = publish(c, 0);
    if (!rc) rc = cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    return rc;
}

int lisa_corrector_forward(const lisa_corrector* c, const float* feats, int64_t M, float* out, void* stream)
{
    if (!c || M < 0 || (M > 0 && (!feats || !out))) { set_error("lisa_corrector_forward: bad arguments"); return LISA_EINVAL; }
    if (((uintptr_t)feats & 15) != 0) { set_error("lisa_corrector_forward: feats must be 16-byte aligned"); return LISA_EINVAL; }
    return run_mlp_tc(c, M, feats, out, nullptr, nullptr, (cudaStream_t)stream);
}

int lisa_corrector_gradient(lisa_corrector* c, const float* feats, const float* target, int64_t n_data,
                            int64_t batch, uint64_t seed, float* grad, float* loss, void* stream)
{
    if (!c || n_data <= 0 || batch < 0 || !feats || !target || !grad) {
        set_error("lisa_corrector_gradient: bad arguments");
        return LISA_EINVAL;
    }
    if (((uintptr_t)feats & 15) != 0) { set_error("lisa_corrector_gradient: feats must be 16-byte aligned"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    int nblk = 0;
    LISA_TRY(run_train_tc(c, feats, target, n_data, batch, seed, &nblk, st));
    prof_before("mlp_grad_reduce", st);
    grad_reduce_kernel<<<(unsigned)((kNParams + 1 + 255) / 256), 256, 0, st>>>(c->part, nblk, grad, loss);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "grad_reduce_kernel launch");
}

int lisa_corrector_adam_step(lisa_corrector* c, const float* grad, float lr, void* stream)
{
    if (!c || !grad || !(lr > 0.f)) { set_error("lisa_corrector_adam_step: bad arguments"); return LISA_EINVAL; }
    return adam_launch(c, grad, 0, nullptr, lr, (cudaStream_t)stream);
}

int lisa_corrector_train(lisa_corrector* c, const float* feats, const float* target, int64_t n_data, int64_t steps,
                         int64_t batch, float lr_max, float lr_min, uint64_t seed, float* losses, void* stream)
{
    if (!c || !feats || !target || n_data <= 0 || steps < 0 || batch <= 0 || !(lr_max > 0.f) || !(lr_min > 0.f) ||
        lr_min > lr_max) {
        set_error("lisa_corrector_train: bad arguments");
        return LISA_EINVAL;
    }
    if (((uintptr_t)feats & 15) != 0) { set_error("lisa_corrector_train: feats must be 16-byte aligned"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t k = 0; k < steps; ++k) {
        // cosine decay from lr_max to lr_min; the Adam kernel sums the partials
        const double lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + cos(M_PI * (double)k / (double)steps));
        int nblk = 0;
        LISA_TRY(run_train_tc(c, feats, target, n_data, batch, seed + ((uint64_t)k << 32), &nblk, st));
        LISA_TRY(adam_launch(c, nullptr, nblk, losses ? losses + k : nullptr, (float)lr, st));
    }
    return LISA_OK;
}

int lisa_corrector_features(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid g, const float* z,
                            const double* y_full, const double* z_ref, double f_lo, double f_hi, float* feats,
                            float* scale, float* ybase, float* target, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(g, "grid"));
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (!(f_lo >= 0.0) || !(f_hi > f_lo)) { set_error("need 0 <= f_lo < f_hi"); return LISA_EINVAL; }
    if (g.n == 0) return LISA_OK;
    if (!z || !feats || !scale || (target && !y_full)) { set_error("NULL series pointer"); return LISA_EINVAL; }
    if (((uintptr_t)feats & 15) != 0) { set_error("feats must be 16-byte aligned"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, g, sc, tab, st));
    return run_features(tab, make_sky_dev(*sky), orbit->L_m / kC, g.dt, z, g.n, g.n, g.n, f_lo, f_hi, feats, scale,
                        ybase, nullptr, 0, g.n, y_full, z_ref, target, st);
}

int lisa_corrector_links(lisa_corrector* c, const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                         const void* hp, const void* hc, lisa_grid out, void* y, void* stream)
{
    if (!c) { set_error("corrector is NULL"); return LISA_EINVAL; }
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(LISA_MIXED, LISA_TDI15, LISA_XYZ));
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!y || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, out, sc, tab, st));
    return corrected_links(c, orbit, sky, h_grid, hp, hc, out, tab, out.n, (float*)y, sc, st);
}

int lisa_response_hybrid_corrected(lisa_corrector* c, const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                                   const void* hp, const void* hc, int tdi_gen, int channels, double t_lo,
                                   double t_hyb, double T_win, double sigma, lisa_grid out, void* xyz, void* stream)
{
    if (!c) { set_error("corrector is NULL"); return LISA_EINVAL; }
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(LISA_MIXED, tdi_gen, channels));
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (!isfinite(t_hyb)) { set_error("t_hyb must be finite"); return LISA_EINVAL; }
    if (isnan(t_lo) || t_lo == INFINITY || t_lo > t_hyb) {
        set_error("t_lo must be -INFINITY or a finite time <= t_hyb");
        return LISA_EINVAL;
    }
    if (out.n == 0) return LISA_OK;
    if (!xyz || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    const double Tw = T_win > 0.0 ? T_win : 800.0 * out.dt;
    const double sg = sigma > 0.0 ? sigma : Tw / 40.0;
    const int64_t n = out.n;
    // plain LFA on [0, iLa], corrected links on [iFa, iLb], full on [iFb, n)
    int64_t iLa = -1, iFa = 0, iLb, iFb;
    if (isfinite(t_lo)) hybrid_split(out, t_lo, Tw, iLa, iFa);
    hybrid_split(out, t_hyb, Tw, iLb, iFb);
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    const SkyDev skyd = make_sky_dev(*sky);
    const double Dmax = 8.0 * max_light_time(orbit, out);
    const int64_t reach = (int64_t)ceil(Dmax / out.dt) + 40;   // TDI delays + stencil, backwards
    // corrected links on the sub-grid [r0, n) of samples [r0, r1): those the TDI
    // of the corrected zone reaches (delays backwards, stencil 16 samples forwards)
    const bool corr_zone = iLb >= iFa;
    const int64_t r0 = corr_zone && iFa - reach > 0 ? iFa - reach : 0;
    const int64_t r1 = iLb + 1 + 32 < n ? iLb + 1 + 32 : n;
    const lisa_grid sub{out.t0 + (double)r0 * out.dt, out.dt, n - r0};
    SegTable tab, tab_sub;
    if (corr_zone) LISA_TRY(make_table_pair(orbit, out, sub, sc, tab, tab_sub, st));
    else LISA_TRY(make_table(orbit, out, sc, tab, st));
    if (iFb > iLb + 1) {
        for (int ch = 0; ch < 3; ++ch) {
            LISA_TRY(cuda_status(cudaMemsetAsync((float*)xyz + (size_t)ch * n + (size_t)(iLb + 1), 0,
                                                 sizeof(float) * (size_t)(iFb - iLb - 1), st), "cudaMemsetAsync"));
        }
    }
    // the full-response links of step 3 depend only on the table and h: they
    // run on a side stream beside steps 1 and 2, joined before step 3's TDI
    float* y = nullptr;
    int64_t lo = 0;
    if (iFb < n) {
        lo = iFb - reach > 0 ? iFb - reach : 0;
        y = (float*)sc.alloc(sizeof(float) * 6 * (size_t)(n - lo));
        if (!y) return sc.status();
    }
    SideGuard side{(iFb < n && (iLa >= 0 || corr_zone)) ? side_acquire() : nullptr};
    int rc_links = 0, rc_join = 0;
    if (side.r) {
        LISA_TRY(cuda_status(cudaEventRecord(side.r->fork, st), "cudaEventRecord"));
        LISA_TRY(cuda_status(cudaStreamWaitEvent(side.r->s, side.r->fork, 0), "cudaStreamWaitEvent"));
        rc_links = launch_links_full(tab, skyd, h_grid, hp, hc, LISA_MIXED, out, y, lo, n, side.r->s, lo);
        rc_join = cuda_status(cudaEventRecord(side.r->join, side.r->s), "cudaEventRecord");
    }
    // steps 1 and 2 on the caller's stream; it joins the side stream afterwards
    // (also after an error, so that nothing queued there outlives the scratch)
    int rc = rc_links ? rc_links : rc_join;
    // 1. plain LFA channels below the lower seam, weight S(t; t_lo, +)
    if (!rc && iLa >= 0) {
        BlendSpec bl{1, t_lo, sg, +1.0, 0, 0};
        rc = launch_lfa(tab, skyd, orbit->L_m, h_grid, hp, hc, LISA_MIXED, tdi_gen, LISA_LFA_UNEQUAL, channels, out,
                        nullptr, xyz, 0, iLa + 1, bl, st);
    }
    // 2. TDI of the corrected links on [iFa, iLb]: weight S(t; t_lo, -) added to
    //    the plain LFA over the lower window; the links are laid out as the TDI
    //    reads samples [r0, n) of the output grid.
    if (!rc && corr_zone) {
        float* yc = (float*)sc.alloc(sizeof(float) * 6 * (size_t)(n - r0));
        rc = yc ? corrected_links(c, orbit, sky, h_grid, hp, hc, sub, tab_sub, r1 - r0, yc, sc, st) : sc.status();
        if (!rc) {
            BlendSpec bl{};
            if (iLa >= 0) bl = BlendSpec{1, t_lo, sg, -1.0, iFa, iLa + 1};
            rc = launch_tdi(tab, out, yc, LISA_MIXED, tdi_gen, LISA_FROZEN, channels, out, xyz, iFa, iLb + 1, bl, st, r0);
        }
    }
    if (side.r && !rc_join) rc_join = cuda_status(cudaStreamWaitEvent(st, side.r->join, 0), "cudaStreamWaitEvent");
    if (rc) return rc;
    if (rc_join) return rc_join;
    // 3. full response above the upper seam: S(t; t_hyb, -) x + (1 - S) out
    //    over the upper window, so that the three weights sum to one
    if (iFb < n) {
        if (!side.r) LISA_TRY(launch_links_full(tab, skyd, h_grid, hp, hc, LISA_MIXED, out, y, lo, n, st, lo));
        BlendSpec bl{1, t_hyb, sg, -1.0, iFb, iLb + 1, 1};
        LISA_TRY(launch_tdi(tab, out, y, LISA_MIXED, tdi_gen, LISA_FROZEN, channels, out, xyz, iFb, n, bl, st, lo));
    }
    return LISA_OK;
}

int lisa_corrector_report(lisa_corrector* c, int64_t* spot_tiles, int64_t* spot_failed, int64_t* band_tiles,
                          int64_t* fallback_tiles, float* max_spot_err, int reset)
{
    if (!c) { set_error("corrector is NULL"); return LISA_EINVAL; }
    CorrStats h;
    LISA_TRY(cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize"));
    LISA_TRY(cuda_status(cudaMemcpy(&h, c->stats, sizeof(h), cudaMemcpyDeviceToHost), "cudaMemcpy"));
    if (spot_tiles) *spot_tiles = h.spot_tiles;
    if (spot_failed) *spot_failed = h.spot_failed;
    if (band_tiles) *band_tiles = h.band_tiles;
    if (fallback_tiles) *fallback_tiles = h.fallback_tiles;
    if (max_spot_err) {
        float e;
        memcpy(&e, &h.max_err_bits, sizeof(e));
        *max_spot_err = e;
    }
    if (reset) LISA_TRY(cuda_status(cudaMemset(c->stats, 0, sizeof(CorrStats)), "cudaMemset"));
    if (h.spot_failed > 0) {
        set_error("%u of %u spot-checked tiles exceeded the tolerance: the full links were used instead",
                  h.spot_failed, h.spot_tiles);
        return LISA_ECORRECTOR;
    }
    return LISA_OK;
}

}  // extern "C"
