// Split-precision products A B^T on tcgen05 tensor cores.
//
// Error-free slicing (after Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012): each row r of an operand is
// scaled by sigma_r = 2^E_r > max |x_r.|, rounded to a fixed-point integer V,
// and V is cut into signed digits that are exact bf16 values:
//     x / sigma = d0 2^-6 + d1 w1 + d2 w2 + ...,  |d0| <= 64,
// with trailing digits of 9 bits (|d| <= 256, w_t = 2^(-6-9t), the per-step
// scheme) or 7 bits (|d| <= 64, w_t = 2^(-6-7t), the accurate scheme).
// A slice product d_s d_t w_s w_t is exact in bf16 x bf16; the products of
// level l = s + t share a TMEM accumulator (levels 0, 1, 2 and >= 3).  Level 0
// sums K <= 4096 products of at most 2^12 units, so its fp32 sum is exact in
// any order; the other levels round far below the slice residuals.  The
// epilogue combines the levels as a two-float (hi = level 0, lo = the rest)
// and scales by sigma_A,i sigma_B,j.
//
// Kernel shape: persistent, one CTA per SM, 10 warps, 128 x 128 output tiles:
//   warp 0  TMA producer (one thread): a ring of STAGES stages, each holding
//           the SA slices of a 128 x 32 A tile and the SB slices of a 128 x 32
//           B tile (64-byte swizzled rows; one 3-D box per operand and stage,
//           {32 k, 128 rows, planes}, the planes 8 KB apart),
//   warp 1  TMEM allocator + MMA issuer (one thread): 2 x pairs tcgen05.mma
//           per stage into the four accumulators (512 TMEM columns),
//   warps 2-9 epilogue, two warps per TMEM lane quadrant, each on 64 columns:
//           they copy the accumulators into registers and release TMEM at
//           once, so the next tile's MMAs run while they scale and store.
// Both operands are K-major (row-major with K contiguous):
//   C[i][j] = sum_k A[i][k] B[j][k].
#include "dme_internal.h"
#include "split_internal.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace dme {

using namespace tc;

constexpr int OZ_BM = 128, OZ_BN = 128, OZ_BK = 32;
constexpr int OZ_SLICE_BYTES = OZ_BM * OZ_BK * 2;                 // 8 KB per slice tile
constexpr int OZ_NACC = 4;                                        // accumulators: levels 0, 1, 2, >= 3
constexpr uint64_t OZ_TIMEOUT_NS = 2000000000ull;                 // 2 s per wait
constexpr int OZ_EPI_WARPS = 8;                                  // two per TMEM lane quadrant
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;               // producer + MMA warps + epilogue
constexpr int OZ_EPI_COLS = OZ_BN / (OZ_EPI_WARPS / 4);          // columns per epilogue warp (64)
constexpr uint32_t OZ_IDESC = idesc_bf16_f32(OZ_BM, OZ_BN);

// Epilogue staging buffer: 32 tile columns x 128 rows of 8-byte outputs (row
// stride 129 words), through which the epilogue writes row segments coalesced.
constexpr int OZ_EPI_STAGE_BYTES = 32 * (OZ_BM + 1) * 8;

template <int SA_, int SB_, int L_, int STAGES_, bool ACC_, int NACC_ = 4>
struct OzCfg {
    static constexpr int SA = SA_, SB = SB_, L = L_, STAGES = STAGES_;
    static constexpr bool ACC = ACC_;                                // accurate mode (exact chunks)
    // TMEM accumulators: levels 0, 1, 2, >= 3 (4), or level 0 and levels >= 1 (2: products
    // of at most 64 K, where the shared accumulator rounds at most four times)
    static constexpr int NACC = NACC_;
    static constexpr int TMEM_COLS = NACC * OZ_BN;
    static constexpr int MIN_BLOCKS = NACC == 2 ? 2 : 1;            // CTAs per SM the registers allow
    static constexpr int A_BYTES = SA * OZ_SLICE_BYTES;
    static constexpr int STAGE_BYTES = (SA + SB) * OZ_SLICE_BYTES;
    // the staged epilogue when the buffer fits beside the stage ring
    static constexpr bool STAGED_EPI = !ACC && STAGES * STAGE_BYTES + OZ_EPI_STAGE_BYTES + 1024 + 256 <= 232448;
    static constexpr int EPI_BYTES = STAGED_EPI ? OZ_EPI_STAGE_BYTES : 0;
    static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024 + 256;
};
using CfgP10 = OzCfg<4, 4, 3, 3, false>;
using CfgP13 = OzCfg<4, 4, 4, 3, false>;
// short products (K <= 64: the Riccati update P - t Y Y^T): one stage, two accumulators,
// 256 TMEM columns and about 100 KB of shared memory, so two CTAs share an SM and their
// epilogues (which are the work here) overlap
// 14 products for at most one wave of tiles (latency-bound, nothing to overlap the epilogue
// with): two stages, so that the staged epilogue fits beside them (same arithmetic as CfgP14)
using CfgP14e = OzCfg<5, 4, 4, 2, false>;
using CfgP10s = OzCfg<4, 4, 3, 1, false, 2>;
using CfgP13s = OzCfg<4, 4, 4, 1, false, 2>;
using CfgP14s = OzCfg<5, 4, 4, 1, false, 2>;
using CfgP14 = OzCfg<5, 4, 4, 3, false>;
using CfgA21 = OzCfg<6, 6, 5, 2, true>;
static_assert(CfgP14::SMEM <= 232448 && CfgA21::SMEM <= 232448, "shared memory per CTA");
static_assert(2 * CfgP14s::SMEM <= 232448 && 2 * CfgP10s::SMEM <= 232448, "two short CTAs per SM");
static_assert(CfgP14e::STAGED_EPI, "the two-stage 14-product form stages its epilogue");

int oz_cfg_pairs(int cfg) {
    switch (cfg) {
        case OZ_P10: return 10;
        case OZ_P13: return 13;
        case OZ_P14: return 14;
        case OZ_A21: return 21;
    }
    return 0;
}
int oz_cfg_slices_a(int cfg) { return cfg == OZ_P14 ? 5 : (cfg == OZ_A21 ? 6 : 4); }
int oz_cfg_slices_b(int cfg) { return cfg == OZ_A21 ? 6 : 4; }
int oz_cfg_scheme(int cfg) { return cfg == OZ_A21 ? OZ_DIG7 : OZ_DIG9; }

// ============================================================== slicing
__device__ __forceinline__ long long round_shift(unsigned long long mag, int shift) {
    if (shift >= 64) return 0;
    if (shift <= 0) return (long long)(mag << (-shift));
    return (long long)((mag + (1ull << (shift - 1))) >> shift);
}

// round(x 2^(B - E)) for a double x with |x| < 2^E (so |result| <= 2^B)
__device__ __forceinline__ long long fixed_d(double x, int E, int B) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF) return 0;
    const unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const long long v = round_shift(M, 1075 - B + E - ex);
    return (b >> 63) ? -v : v;
}

// round(f 2^(B - E)) for a float f
__device__ __forceinline__ long long fixed_f(float f, int E, int B) {
    const unsigned int b = __float_as_uint(f);
    const int ef = (int)((b >> 23) & 0xFF);
    if (ef == 0 || ef == 0xFF) return 0;
    const unsigned long long M = (b & 0x7FFFFFu) | 0x800000u;
    const long long v = round_shift(M, 150 - B + E - ef);
    return (b >> 31) ? -v : v;
}

// Fixed-point width B of a scheme: the leading digit has weight 2^-6, the last
// representable one 2^-B (DIG9: 6 + 4 x 9 = 42 bits, DIG7: 6 + 5 x 7 = 41 bits).
template <int SCHEME>
struct Digits {
    static constexpr int B = SCHEME == OZ_DIG9 ? 42 : 41;
    static constexpr int TOP = B - 6;                    // shift of digit 0
};

// The NS leading digits of V (|V| < 2^B), each rounded to nearest:
// d_t = round(r_t / 2^(TOP - b t)), r_{t+1} = r_t - d_t 2^(TOP - b t); the last
// digit absorbs (rounds) whatever lies below it.
template <int SCHEME, int NS>
__device__ __forceinline__ void digits(long long V, int (&dg)[NS]) {
    constexpr int b = SCHEME;
    long long r = V;
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        const int sh = Digits<SCHEME>::TOP - b * t;
        if (sh <= 0) {
            dg[t] = (int)r;
            r = 0;
        } else {
            const long long d = (r + (1ll << (sh - 1))) >> sh;
            dg[t] = (int)d;
            r -= d << sh;
        }
    }
}

template <int SCHEME>
__device__ __forceinline__ float digit_unit(int t) {
    return __int_as_float((127 - 6 - SCHEME * t) << 23);      // 2^(-6 - b t), exact
}

// Load entries k .. k+3 of a row (zeros past `cols`); vector loads when the
// row start is 16-byte aligned and the four entries are in range.
template <bool PAIR>
__device__ __forceinline__ void load4(const double* X, const float2* Xp, size_t base, int k, int cols, bool vec,
                                      double (&d)[4], float2 (&f)[4]) {
    if (vec && k + 3 < cols) {
        if (PAIR) {
            const float4 a = *reinterpret_cast<const float4*>(Xp + base + k);
            const float4 b = *reinterpret_cast<const float4*>(Xp + base + k + 2);
            f[0] = make_float2(a.x, a.y);
            f[1] = make_float2(a.z, a.w);
            f[2] = make_float2(b.x, b.y);
            f[3] = make_float2(b.z, b.w);
        } else {
            const double2 a = *reinterpret_cast<const double2*>(X + base + k);
            const double2 b = *reinterpret_cast<const double2*>(X + base + k + 2);
            d[0] = a.x;
            d[1] = a.y;
            d[2] = b.x;
            d[3] = b.y;
        }
    } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (PAIR) f[u] = (k + u < cols) ? Xp[base + k + u] : make_float2(0.f, 0.f);
            else d[u] = (k + u < cols) ? X[base + k + u] : 0.0;
        }
    }
}

template <bool PAIR>
__device__ __forceinline__ int entry_exp(const double& d, const float2& f) {
    if (PAIR) {
        const unsigned int b = __float_as_uint(f.x) & 0x7FFFFFFFu;
        const int ef = (int)(b >> 23);
        return (b == 0 || ef == 0) ? -100000 : ef - 127;
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int ed = (int)((b >> 52) & 0x7FF);
    return (ed == 0) ? -100000 : ed - 1023;
}

// Write the NS slices of four consecutive entries (fixed-point values V) at
// plane offset o: one 8-byte store of four bf16 per plane.
template <int SCHEME, int NS>
__device__ __forceinline__ void store_slices4(const long long (&V)[4], __nv_bfloat16* __restrict__ out, size_t o,
                                              size_t plane) {
    int dg[4][NS];
#pragma unroll
    for (int u = 0; u < 4; ++u) digits<SCHEME, NS>(V[u], dg[u]);
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        const float unit = digit_unit<SCHEME>(t);
        float q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = (float)dg[u][t] * unit;      // |d| <= 256: exact in bf16
        const __nv_bfloat162 p01 = __floats2bfloat162_rn(q[0], q[1]);
        const __nv_bfloat162 p23 = __floats2bfloat162_rn(q[2], q[3]);
        uint2 w;
        w.x = *reinterpret_cast<const unsigned int*>(&p01);
        w.y = *reinterpret_cast<const unsigned int*>(&p23);
        *reinterpret_cast<uint2*>(out + t * plane + o) = w;
    }
}

template <bool PAIR, int SCHEME>
__device__ __forceinline__ long long to_fixed(const double& d, const float2& f, int E) {
    constexpr int B = Digits<SCHEME>::B;
    return PAIR ? fixed_f(f.x, E, B) + fixed_f(f.y, E, B) : fixed_d(d, E, B);
}

// One warp per row: pass 1 finds the row's max exponent, pass 2 writes the
// NS slices (zero beyond `cols`, up to Kp) and the row scale 2^E.
template <bool PAIR, int SCHEME, int NS>
__device__ __forceinline__ void slice_row_warp(const double* __restrict__ X, const float2* __restrict__ Xp, int row,
                                               int cols, int ldx, __nv_bfloat16* __restrict__ out, int Kp,
                                               float* __restrict__ scale, int prow) {
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)row * ldx;
    const bool vec = (ldx % 2) == 0;
    double d[4];
    float2 f[4];
    int emax = -100000;
    for (int k = 4 * lane; k < cols; k += 128) {
        load4<PAIR>(X, Xp, base, k, cols, vec, d, f);
#pragma unroll
        for (int u = 0; u < 4; ++u) emax = max(emax, entry_exp<PAIR>(d[u], f[u]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    // rows whose largest entry is below 2^-100 or above 2^126 are stored as zero
    // (fp32 scales and products must stay normal)
    const bool zero_row = emax < -100 || emax > 126;
    const int E = emax + 1;                       // |x| < 2^E for every entry of the row
    if (lane == 0) scale[row] = zero_row ? 0.0f : ldexpf(1.0f, E);
    const size_t plane = (size_t)prow * Kp;     // planes hold prow >= rows rows
    for (int k = 4 * lane; k < Kp; k += 128) {
        long long V[4] = {0, 0, 0, 0};
        if (!zero_row && k < cols) {
            load4<PAIR>(X, Xp, base, k, cols, vec, d, f);
#pragma unroll
            for (int u = 0; u < 4; ++u) V[u] = to_fixed<PAIR, SCHEME>(d[u], f[u], E);
        }
        store_slices4<SCHEME, NS>(V, out, (size_t)row * Kp + k, plane);
    }
}

template <bool PAIR, int SCHEME, int NS>
__global__ void __launch_bounds__(256) slice_rows_kernel(const double* __restrict__ X, const float2* __restrict__ Xp,
                                                         int rows, int cols, int ldx, __nv_bfloat16* __restrict__ out,
                                                         int Kp, float* __restrict__ scale, int prow) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= rows) return;
    slice_row_warp<PAIR, SCHEME, NS>(X, Xp, row, cols, ldx, out, Kp, scale, prow);
}

// Grouped slicing (serving): the rows of several problems laid end to end,
// a warp per row; warp w finds its problem by a binary search over row0.
template <bool PAIR>
__global__ void __launch_bounds__(256) slice_rows_grouped_kernel(const SliceDesc* __restrict__ d, int nd,
                                                                 int total_rows) {
    const int g = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (g >= total_rows) return;
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].row0 <= g) lo = mid;
        else hi = mid - 1;
    }
    const SliceDesc& q = d[lo];
    slice_row_warp<PAIR, OZ_DIG9, 4>(q.X, q.Xp, g - q.row0, q.cols, q.ldx, q.out, q.Kp, q.scale, q.prow);
}

// Long rows (Kp > 1024): one CTA of 256 threads per row; each thread keeps G
// groups of 4 consecutive entries (k = 4 tid + 1024 g) in registers, so the
// row is read from memory once; the row maximum is a block reduction.  Same
// digits as slice_rows_kernel.
template <bool PAIR, int SCHEME, int NS, int G>
__global__ void __launch_bounds__(256) slice_long_rows_kernel(const double* __restrict__ X,
                                                              const float2* __restrict__ Xp, int rows, int cols,
                                                              int ldx, __nv_bfloat16* __restrict__ out, int Kp,
                                                              float* __restrict__ scale, int prow) {
    __shared__ int wmax[8];
    const int row = blockIdx.x, tid = threadIdx.x;
    const size_t base = (size_t)row * ldx;
    const bool vec = (ldx % 2) == 0;
    double d[G][4];
    float2 f[G][4];
    int emax = -100000;
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int k = 4 * tid + 1024 * g;
        if (k < cols) {
            load4<PAIR>(X, Xp, base, k, cols, vec, d[g], f[g]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                d[g][u] = 0.0;
                f[g][u] = make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) emax = max(emax, entry_exp<PAIR>(d[g][u], f[g][u]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    if ((tid & 31) == 0) wmax[tid >> 5] = emax;
    __syncthreads();
    emax = wmax[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) emax = max(emax, wmax[w]);
    const bool zero_row = emax < -100 || emax > 126;
    const int E = emax + 1;
    if (tid == 0) scale[row] = zero_row ? 0.0f : ldexpf(1.0f, E);
    const size_t plane = (size_t)prow * Kp;     // planes hold prow >= rows rows
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int k = 4 * tid + 1024 * g;
        if (k >= Kp) continue;
        long long V[4] = {0, 0, 0, 0};
        if (!zero_row && k < cols) {
#pragma unroll
            for (int u = 0; u < 4; ++u) V[u] = to_fixed<PAIR, SCHEME>(d[g][u], f[g][u], E);
        }
        store_slices4<SCHEME, NS>(V, out, (size_t)row * Kp + k, plane);
    }
}

template <bool PAIR, int SCHEME, int NS>
static void slice_launch(const double* X, const float2* Xp, int rows, int cols, int ldx, const SliceBuf& sb,
                         cudaStream_t st) {
    if (rows <= 0 || rows > sb.rows) return;
    const int pr = sb.rows;
    if (sb.Kp > 2048)
        slice_long_rows_kernel<PAIR, SCHEME, NS, 4>
            <<<rows, 256, 0, st>>>(X, Xp, rows, cols, ldx, sb.data, sb.Kp, sb.scale, pr);
    else if (sb.Kp > 1024)
        slice_long_rows_kernel<PAIR, SCHEME, NS, 2>
            <<<rows, 256, 0, st>>>(X, Xp, rows, cols, ldx, sb.data, sb.Kp, sb.scale, pr);
    else
        slice_rows_kernel<PAIR, SCHEME, NS>
            <<<(rows + 7) / 8, 256, 0, st>>>(X, Xp, rows, cols, ldx, sb.data, sb.Kp, sb.scale, pr);
}

dme_status launch_slice_grouped(std::vector<SliceDesc>& items, bool pair, cudaStream_t st, DescArena* arena) {
    int total = 0;
    for (auto& it : items) {
        if (it.ns != 4 || it.rows <= 0) return set_error("grouped slicing: 4 slices and rows > 0"), DME_EINVAL;
        it.row0 = total;
        total += it.rows;
    }
    if (total == 0) return DME_OK;
    const SliceDesc* dd = static_cast<const SliceDesc*>(arena->put(items.data(), items.size() * sizeof(SliceDesc)));
    if (!dd) return set_error("grouped slicing: descriptor arena full"), DME_ENOMEM;
    const int grid = (total + 7) / 8;
    if (pair) slice_rows_grouped_kernel<true><<<grid, 256, 0, st>>>(dd, (int)items.size(), total);
    else slice_rows_grouped_kernel<false><<<grid, 256, 0, st>>>(dd, (int)items.size(), total);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

void launch_slice_rows_f64(const double* X, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st) {
    if (sb.scheme == OZ_DIG7) slice_launch<false, OZ_DIG7, 6>(X, nullptr, rows, cols, ldx, sb, st);
    else if (sb.ns == 5) slice_launch<false, OZ_DIG9, 5>(X, nullptr, rows, cols, ldx, sb, st);
    else slice_launch<false, OZ_DIG9, 4>(X, nullptr, rows, cols, ldx, sb, st);
}

void launch_slice_rows_pair(const float2* Xp, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st) {
    if (sb.ns == 5) slice_launch<true, OZ_DIG9, 5>(nullptr, Xp, rows, cols, ldx, sb, st);
    else slice_launch<true, OZ_DIG9, 4>(nullptr, Xp, rows, cols, ldx, sb, st);
}

// ============================================================== tcgen05 GEMM
// Tile order.  Tiles run in groups of OZ_GROUP tile rows, column by column
// inside a group, so the CTAs working at one time touch the group's row tiles
// of A (8 x 128 rows) and about 152/OZ_GROUP column tiles of B, which stay in
// L2; B is read once per group.  Triangle grids do the same over the tiles
// with tm <= tn.  (Groups of 16 measured 1 % slower at n = 4096.)
constexpr int OZ_GROUP = 8;

__device__ __forceinline__ void oz_tile_coords(const OzParams& p, int t, int& tm, int& tn) {
    if (p.tri) {
        // group g holds rows [8 g, 8 g + 8); its column tn carries the rows tm <= tn
        const int T = p.tiles_n;
        int first = 0, rem = t;
        while (true) {
            const int rows = min(OZ_GROUP, T - first);
            // tiles of the group: columns first .. first+rows-1 carry 1 .. rows, the rest rows each
            const int in_group = rows * (rows + 1) / 2 + rows * (T - first - rows);
            if (rem < in_group) {
                int c = first;
                while (true) {
                    const int cnt = min(c - first + 1, rows);
                    if (rem < cnt) {
                        tm = first + rem;
                        tn = c;
                        return;
                    }
                    rem -= cnt;
                    ++c;
                }
            }
            rem -= in_group;
            first += rows;
        }
    } else {
        const int tiles_m = (p.M + 127) / 128;
        const int per_group = OZ_GROUP * p.tiles_n;
        const int g = t / per_group;
        const int first = g * OZ_GROUP;
        const int rows = min(OZ_GROUP, tiles_m - first);
        const int r = t - g * per_group;
        tm = first + r % rows;
        tn = r / rows;
    }
}

// Exact float -> double conversion of a normal or zero float by bit moves
// (subnormal floats are flushed to zero; the epilogue never produces them
// for in-range data).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int e = (b >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    const unsigned long long ed = (unsigned long long)(e - 127 + 1023) << 52;
    const unsigned long long m = (unsigned long long)(b & 0x7FFFFFu) << 29;
    return __longlong_as_double((long long)(sign | ed | m));
}

// What one work unit of a launch is: a 128 x 128 output tile of one problem
// over the K blocks [kb0, kb0 + nk), as part `part` of `nparts` (split K of the
// tail; widx = its workspace slot) or as accurate-mode chunk `chunk`.
struct OzUnit {
    const OzParams* p;
    const CUtensorMap* tA;
    const CUtensorMap* tB;
    int tm, tn, kb0, nk, part, nparts, widx, chunk;
};

__device__ __forceinline__ void oz_single_unit(const OzParams* p, const CUtensorMap* tA, const CUtensorMap* tB,
                                               bool acc, int u, OzUnit& o) {
    o.p = p;
    o.tA = tA;
    o.tB = tB;
    const int nk_all = p->Kp / OZ_BK;
    int tile = u, part = 0, nparts = 1, widx = 0, chunk = 0;
    if (acc) {
        // chunk-major: the units working at one time share one K range
        chunk = u / p->tiles;
        tile = u - chunk * p->tiles;
    } else if (p->split_parts > 1 && u >= p->split_first) {
        const int j = u - p->split_first;
        tile = p->split_first + j / p->split_parts;
        part = j % p->split_parts;
        nparts = p->split_parts;
        widx = j / p->split_parts;
    }
    oz_tile_coords(*p, tile, o.tm, o.tn);
    if (acc) {
        o.kb0 = chunk * OZ_ACC_CHUNK_KB;
        o.nk = min(OZ_ACC_CHUNK_KB, nk_all - o.kb0);
    } else {
        o.kb0 = part * nk_all / nparts;
        o.nk = (part + 1) * nk_all / nparts - o.kb0;
    }
    o.part = part;
    o.nparts = nparts;
    o.widx = widx;
    o.chunk = chunk;
}

__device__ __forceinline__ void oz_group_unit(const OzGroupDesc* __restrict__ d, int nd, int u, OzUnit& o) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].start <= u) lo = mid;
        else hi = mid - 1;
    }
    oz_single_unit(&d[lo].p, &d[lo].tmA, &d[lo].tmB, false, u - d[lo].start, o);
}

// Load 32 columns of the four accumulators of TMEM lane quadrant q at column c0
// into h (level 0, raw fp32 bits) and l (levels 1 + 2 + 3.., as fp32 bits).
// (The levels 2 and 3 come through a 16-column temporary: the epilogue warps
// hold 128 values each and the kernel's register budget is 168.)
__device__ __forceinline__ void oz_load_half(uint32_t tmem, int q, int c0, uint32_t (&h)[32], uint32_t (&l)[32]) {
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0;
    tmem_ld_32x32b_x32(ta, h);
    tmem_ld_32x32b_x32(ta + OZ_BN, l);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        uint32_t t[16];
        tmem_ld_32x32b_x16(ta + 2 * OZ_BN + 16 * g, t);
        tmem_ld_wait();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
            l[16 * g + jj] = __float_as_uint(__uint_as_float(l[16 * g + jj]) + __uint_as_float(t[jj]));
        tmem_ld_32x32b_x16(ta + 3 * OZ_BN + 16 * g, t);
        tmem_ld_wait();
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
            l[16 * g + jj] = __float_as_uint(__uint_as_float(l[16 * g + jj]) + __uint_as_float(t[jj]));
    }
}

// Epilogue of 32 columns (tile columns c0 .. c0+31) of row i from registers.
__device__ __forceinline__ void oz_store_half(const OzParams& p, int m0, int n0, int i, int c0, bool diag,
                                              const uint32_t (&h)[32], const uint32_t (&l)[32]) {
    if (i >= p.M) return;
    const float sA = p.sa[i];
    if (p.mode == OZ_OUT_PAIR) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
            const int j = n0 + c0 + jj;
            if (j >= p.N) break;
            const float s = sA * p.sb[j];
            const float hv = __uint_as_float(h[jj]), lv = __uint_as_float(l[jj]);
            // TwoSum: (sh, sl) = hi + lo exactly
            const float sh = hv + lv;
            const float bb = sh - hv;
            const float sl = (hv - (sh - bb)) + (lv - bb);
            p.Cp[(size_t)i * p.ldc + j] = make_float2(sh * s, sl * s);
        }
        return;
    }
    const double alpha = p.alpha;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
        const int j = n0 + c0 + jj;
        if (j >= p.N) break;
        if (diag && i > j) continue;                   // lower half of a diagonal tile: its mirror owns it
        const float s = sA * p.sb[j];
        const float hv = __uint_as_float(h[jj]), lv = __uint_as_float(l[jj]);
        const float sh = hv + lv;
        const float bb = sh - hv;
        const float sl = (hv - (sh - bb)) + (lv - bb);
        double v = f2d_bits(sh * s) + f2d_bits(sl * s);
        if (alpha != 1.0) v *= alpha;
        if (p.tri) {
            // symmetric output and addends: read the addends at (j, i) (coalesced over
            // the warp's rows), write (j, i) and its mirror (i, j)
            const size_t tof = (size_t)j * p.ldc + i;
            if (p.D1) v += p.b1 * p.D1[tof];
            if (p.D2) v += p.b2 * p.D2[tof];
            if (p.D3) v += p.b3 * p.D3[tof];
            p.Cd[tof] = v;
            if (i != j) p.Cd[(size_t)i * p.ldc + j] = v;
        } else {
            const size_t off = (size_t)i * p.ldc + j;
            if (p.D1) v += p.b1 * p.D1[off];
            if (p.D2) v += p.b2 * p.D2[off];
            if (p.D3) v += p.b3 * p.D3[off];
            p.Cd[off] = v;
        }
    }
}

// Staged epilogue of one 16-column round: the thread of tile row il holds the
// level sums of columns c0 + h0 .. c0 + h0 + 15 (entries h0 .. h0 + 15 of h, l).
// Phase 1: each thread forms its 16 outputs (FP64 value or normalised pair);
// a triangle output also goes straight to its mirror (j, i), coalesced over the
// warp's rows, with the symmetric addends read at (j, i); every output is put
// in the staging buffer T (16 columns of the two warps of a lane quadrant, so
// T holds 32 tile columns).  Phase 2: the 256 epilogue threads write the 128
// staged row segments (i, j) coalesced (non-triangle F64 outputs add their
// addends here, read at (i, j)).  Two named-barrier syncs per round.
__device__ __forceinline__ void oz_store_staged(const OzParams& p, int m0, int n0, int il, int c0, int h0, bool diag,
                                                const uint32_t (&h)[32], const uint32_t (&l)[32], uint64_t* T,
                                                int ew, int lane) {
    const int i = m0 + il;
    const int slot = (ew / 4) * 16;                        // T columns of this warp pair: 0..15 or 16..31
    if (i < p.M) {
        const float sA = p.sa[i];
        // four columns at a time: their addends are loaded before any of the four
        // stores (an in-place update may alias Cd and D1, which would otherwise
        // serialise every load behind the previous store)
#pragma unroll
        for (int g = 0; g < 16; g += 4) {
            double a1[4], a2[4], a3[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = n0 + c0 + h0 + g + u;
                const bool in = p.mode == OZ_OUT_F64 && p.tri && j < p.N && !(diag && i > j);
                const size_t tof = (size_t)j * p.ldc + i;
                a1[u] = (in && p.D1) ? p.D1[tof] : 0.0;
                a2[u] = (in && p.D2) ? p.D2[tof] : 0.0;
                a3[u] = (in && p.D3) ? p.D3[tof] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jj = g + u;
                const int j = n0 + c0 + h0 + jj;
                if (j >= p.N) break;
                const float s = sA * p.sb[j];
                const float hv = __uint_as_float(h[h0 + jj]), lv = __uint_as_float(l[h0 + jj]);
                const float sh = hv + lv;
                const float bb = sh - hv;
                const float sl = (hv - (sh - bb)) + (lv - bb);
                uint64_t word;
                if (p.mode == OZ_OUT_PAIR) {
                    const float2 v = make_float2(sh * s, sl * s);
                    word = *reinterpret_cast<const uint64_t*>(&v);
                } else {
                    double v = f2d_bits(sh * s) + f2d_bits(sl * s);
                    if (p.alpha != 1.0) v *= p.alpha;
                    if (p.tri) {
                        if (diag && i > j) continue;           // its mirror (j, i) owns this entry
                        if (p.D1) v += p.b1 * a1[u];
                        if (p.D2) v += p.b2 * a2[u];
                        if (p.D3) v += p.b3 * a3[u];
                        p.Cd[(size_t)j * p.ldc + i] = v;
                    }
                    word = (uint64_t)__double_as_longlong(v);
                }
                T[(slot + jj) * (OZ_BM + 1) + il] = word;
            }
        }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    // phase 2: warp ew writes tile rows 16 ew .. 16 ew + 15; lanes 0-15 the first warp
    // pair's 16 columns (tile columns c0' + h0 ..), lanes 16-31 the second pair's (c0' + 64)
    const int half = lane >> 4, jl = lane & 15;
    const int cbase = (c0 - (ew / 4) * 64) + half * 64 + h0;   // tile column of this lane's slot
    const int j = n0 + cbase + jl;
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
        const int rl = 16 * ew + r;
        const int gi = m0 + rl;
        if (gi >= p.M || j >= p.N) continue;
        if (p.tri && (gi >= j)) continue;            // (i, i) and below: written in phase 1 (or by the mirror)
        const uint64_t word = T[(half * 16 + jl) * (OZ_BM + 1) + rl];
        const size_t off = (size_t)gi * p.ldc + j;
        if (p.mode == OZ_OUT_PAIR) {
            p.Cp[off] = *reinterpret_cast<const float2*>(&word);
        } else {
            double v = __longlong_as_double((long long)word);
            if (!p.tri) {
                if (p.D1) v += p.b1 * p.D1[off];
                if (p.D2) v += p.b2 * p.D2[off];
                if (p.D3) v += p.b3 * p.D3[off];
            }
            p.Cd[off] = v;
        }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

// Accurate-mode epilogue of 32 columns: the levels added in fp64 (levels 0-2
// of a chunk are exact fp32 integers of their units, so the double sum is
// exact but for the shared level-3 accumulator's own rounding), scaled, and
// written to the chunk's slab of the workspace.
__device__ __forceinline__ void oz_store_chunk_half(const OzParams& p, uint32_t tmem, int q, int c0, int m0, int n0,
                                                    int i, int chunk) {
    uint32_t a0[32], a1[32], a2[32], a3[32];
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0;
    tmem_ld_32x32b_x32(ta, a0);
    tmem_ld_32x32b_x32(ta + OZ_BN, a1);
    tmem_ld_32x32b_x32(ta + 2 * OZ_BN, a2);
    tmem_ld_32x32b_x32(ta + 3 * OZ_BN, a3);
    tmem_ld_wait();
    if (i >= p.M) return;
    const double sA = (double)p.sa[i];
    double* out = p.wsd + ((size_t)chunk * p.M + i) * p.N;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
        const int j = n0 + c0 + jj;
        if (j >= p.N) break;
        double v = f2d_bits(__uint_as_float(a0[jj])) + f2d_bits(__uint_as_float(a1[jj]));
        v += f2d_bits(__uint_as_float(a2[jj]));
        v += f2d_bits(__uint_as_float(a3[jj]));
        out[j] = v * (sA * (double)p.sb[j]);
    }
}

// The persistent loop.  Every role walks the same unit sequence
// u = blockIdx.x, blockIdx.x + gridDim.x, ...; `resolve(u, unit)` maps a unit
// index to its problem, tile and K range.
template <class Cfg, class Resolve>
__device__ __forceinline__ void oz_persistent(int units, Resolve resolve) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* stage_T = reinterpret_cast<uint64_t*>(smem + Cfg::STAGES * Cfg::STAGE_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::STAGES * Cfg::STAGE_BYTES + Cfg::EPI_BYTES);
    // bars[0..S): full, [S..2S): empty, [2S]: accumulators full, [2S+1]: accumulators
    // empty, [2S+2]: drain (every MMA done before TMEM is freed)
    constexpr int S = Cfg::STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 3);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[S + s]), 1);
        }
        mbar_init(smem_u32(&bars[2 * S]), 1);
        mbar_init(smem_u32(&bars[2 * S + 1]), OZ_EPI_WARPS);
        mbar_init(smem_u32(&bars[2 * S + 2]), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), Cfg::TMEM_COLS);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t acc_full = smem_u32(&bars[2 * S]), acc_empty = smem_u32(&bars[2 * S + 1]);

    if (warp == 0) {
        if (lane == 0) {
            uint32_t issued = 0, last_ph = 0;               // per stage: a load issued, its phase parity
            int kit = 0;                                    // k blocks issued over all units
            bool ok = true;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                OzUnit w;
                resolve(u, w);
                const OzParams& p = *w.p;
                tma_prefetch_desc(w.tA);
                tma_prefetch_desc(w.tB);
                const int m0 = w.tm * OZ_BM, n0 = w.tn * OZ_BN;
                for (int it = 0; it < w.nk; ++it, ++kit) {
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    const int s = kit % S;
                    const uint32_t ph = (kit / S) & 1;
                    if (kit >= S && !mbar_wait(smem_u32(&bars[S + s]), ph ^ 1, OZ_TIMEOUT_NS)) {
                        atomicOr(p.status, DEV_TIMEOUT);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bars[s]);
                    uint8_t* st = smem + s * Cfg::STAGE_BYTES;
                    const int kc = (w.kb0 + it) * OZ_BK;
                    mbar_arrive_expect_tx(full, Cfg::STAGE_BYTES);
                    // one box per operand: the 32 x 128 tile of each of its SA (SB) planes,
                    // planes 8 KB apart in the stage
                    tma_load_3d(smem_u32(st), w.tA, full, kc, m0, 0);
                    tma_load_3d(smem_u32(st + Cfg::A_BYTES), w.tB, full, kc, n0, 0);
                    issued |= 1u << s;
                    last_ph = (last_ph & ~(1u << s)) | (ph << s);
                    // pull the epilogue's addend rows into L2: spread over the K loop, and all
                    // of them at the last k block of a short one (full 128-column segments
                    // only, 16-byte aligned; transposed for tri outputs)
                    if (!Cfg::ACC && p.mode == OZ_OUT_F64 && (p.ldc % 2) == 0 && (p.D1 || p.D2)) {
                        const int r0 = it, r1 = (it == w.nk - 1) ? OZ_BM : min(it + 1, OZ_BM);
                        for (int rr = r0; rr < r1; ++rr) {
                            const int ra = (p.tri ? n0 : m0) + rr, ca = p.tri ? m0 : n0;
                            const int rmax = p.tri ? p.N : p.M, cmax = p.tri ? p.M : p.N;
                            if (ra >= rmax || ca + OZ_BN > cmax) continue;
                            const size_t off = (size_t)ra * p.ldc + ca;
                            if (p.D1 && ((reinterpret_cast<uintptr_t>(p.D1 + off) & 15) == 0))
                                prefetch_l2_bulk(p.D1 + off, OZ_BN * sizeof(double));
                            if (p.D2 && ((reinterpret_cast<uintptr_t>(p.D2 + off) & 15) == 0))
                                prefetch_l2_bulk(p.D2 + off, OZ_BN * sizeof(double));
                        }
                    }
                }
            }
            // every load this thread issued has landed before the CTA may exit
            for (int s = 0; s < S; ++s)
                if (((issued >> s) & 1u) && !mbar_wait(smem_u32(&bars[s]), (last_ph >> s) & 1u, OZ_TIMEOUT_NS))
                    *abort_flag = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int kit = 0, li = 0;
            int* status = nullptr;
            for (int u = blockIdx.x; u < units; u += gridDim.x, ++li) {
                if (*abort_flag) break;
                OzUnit w;
                resolve(u, w);
                status = w.p->status;
                // the epilogue has copied the previous unit's accumulators out of TMEM
                if (li > 0 && !mbar_wait(acc_empty, (li - 1) & 1, OZ_TIMEOUT_NS)) {
                    atomicOr(status, DEV_TIMEOUT);
                    *abort_flag = 1;
                    break;
                }
                fence_after_sync();
                bool ok = true;
                // the unit's own level cut: a grouped launch of the 4 x 4 slice kernel also
                // runs 10-product problems (levels <= 3), with the same MMAs in the same order
                // as their own kernel
                const int Lu = min(Cfg::L, w.p->cfg == OZ_P10 ? 3 : Cfg::L);
                for (int it = 0; it < w.nk; ++it, ++kit) {
                    const int s = kit % S;
                    const uint32_t ph = (kit / S) & 1;
                    if (!mbar_wait(smem_u32(&bars[s]), ph, OZ_TIMEOUT_NS)) {
                        atomicOr(status, DEV_TIMEOUT);
                        *abort_flag = 1;
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t a0 = smem_u32(smem + s * Cfg::STAGE_BYTES);
                    const uint32_t b0 = a0 + Cfg::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
                        for (int sa = 0; sa < Cfg::SA; ++sa) {
#pragma unroll
                            for (int sb = 0; sb < Cfg::SB; ++sb) {
                                if (sa + sb > Cfg::L || sa + sb > Lu) continue;
                                const int lvl = (sa + sb < Cfg::NACC - 1) ? sa + sb : Cfg::NACC - 1;
                                const uint64_t ad = desc_kmajor_sw64(a0 + sa * OZ_SLICE_BYTES + kk * 32);
                                const uint64_t bd = desc_kmajor_sw64(b0 + sb * OZ_SLICE_BYTES + kk * 32);
                                // the pairs (0, t), t <= 3, come first and open accumulator t at the
                                // unit's first k step; everything else accumulates
                                const uint32_t acc = (it == 0 && kk == 0 && sa == 0 && sb < Cfg::NACC) ? 0u : 1u;
                                mma_bf16(tmem + (uint32_t)(lvl * OZ_BN), ad, bd, OZ_IDESC, acc);
                            }
                        }
                    }
                    mma_commit(smem_u32(&bars[S + s]));
                }
                if (!ok) break;
                mma_commit(acc_full);
            }
            // every MMA issued has completed before TMEM is released
            mma_commit(smem_u32(&bars[2 * S + 2]));
            if (!mbar_wait(smem_u32(&bars[2 * S + 2]), 0, OZ_TIMEOUT_NS)) {
                if (status) atomicOr(status, DEV_TIMEOUT);
                *abort_flag = 1;
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = tile rows, columns
        // [cq, cq + 64) with cq = 64 * ((w - 2) / 4)
        const int q = warp & 3;
        const int ew = warp - 2;                                   // 0 .. OZ_EPI_WARPS-1
        const int cq = OZ_EPI_COLS * (ew / 4);
        int li = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++li) {
            OzUnit w;
            resolve(u, w);
            const OzParams& p = *w.p;
            const bool ready_here = !*abort_flag && mbar_wait(acc_full, li & 1, OZ_TIMEOUT_NS);
            // one decision for all epilogue threads (they share named barrier 1 below)
            uint32_t all_ready;
            asm volatile(
                "{\n"
                " .reg .pred p, r;\n"
                " setp.ne.u32 p, %1, 0;\n"
                " bar.red.and.pred r, 1, 256, p;\n"
                " selp.u32 %0, 1, 0, r;\n"
                "}\n"
                : "=r"(all_ready)
                : "r"((uint32_t)ready_here)
                : "memory");
            if (!all_ready) {
                if (lane == 0) atomicOr(p.status, DEV_TIMEOUT);
                *abort_flag = 1;
                break;
            }
            fence_after_sync();
            const int m0 = w.tm * OZ_BM, n0 = w.tn * OZ_BN;
            const int il = 32 * q + lane;                          // tile row of this thread
            const int i = m0 + il;
            if (Cfg::ACC) {
                oz_store_chunk_half(p, tmem, q, cq, m0, n0, i, w.chunk);
                oz_store_chunk_half(p, tmem, q, cq + 32, m0, n0, i, w.chunk);
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
                continue;
            }
            if (Cfg::NACC == 2) {
                // short products (never split in K): 32 columns at a time, TMEM released at
                // the end (the next unit's product is as short), so that the registers allow
                // two CTAs per SM
                const bool diag = p.tri && w.tm == w.tn;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t hs[32], ls[32];
                    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cq + 32 * hh);
                    tmem_ld_32x32b_x32(ta, hs);
                    tmem_ld_32x32b_x32(ta + OZ_BN, ls);
                    tmem_ld_wait();
                    oz_store_staged(p, m0, n0, il, cq + 32 * hh, 0, diag, hs, ls, stage_T, ew, lane);
                    oz_store_staged(p, m0, n0, il, cq + 32 * hh, 16, diag, hs, ls, stage_T, ew, lane);
                }
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
                continue;
            }
            uint32_t h0[32], l0[32], h1[32], l1[32];
            if (Cfg::NACC == 4) {
                oz_load_half(tmem, q, cq, h0, l0);
                oz_load_half(tmem, q, cq + 32, h1, l1);
            } else {
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cq;
                tmem_ld_32x32b_x32(ta, h0);
                tmem_ld_32x32b_x32(ta + OZ_BN, l0);
                tmem_ld_32x32b_x32(ta + 32, h1);
                tmem_ld_32x32b_x32(ta + OZ_BN + 32, l1);
                tmem_ld_wait();
            }
            // the accumulators are in registers: hand TMEM back to the MMA warp
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
            if (w.nparts > 1) {
                // split K: publish this part's level sums; oz_tail_kernel adds the parts
                constexpr size_t tile_elems = (size_t)OZ_BM * OZ_BN;
                float2* mine = p.ws + ((size_t)w.widx * w.nparts + w.part) * tile_elems + (size_t)il * OZ_BN + cq;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    mine[jj] = make_float2(__uint_as_float(h0[jj]), __uint_as_float(l0[jj]));
                    mine[32 + jj] = make_float2(__uint_as_float(h1[jj]), __uint_as_float(l1[jj]));
                }
                continue;
            }
            const bool diag = p.tri && w.tm == w.tn;
            if (Cfg::STAGED_EPI) {
                oz_store_staged(p, m0, n0, il, cq, 0, diag, h0, l0, stage_T, ew, lane);
                oz_store_staged(p, m0, n0, il, cq, 16, diag, h0, l0, stage_T, ew, lane);
                oz_store_staged(p, m0, n0, il, cq + 32, 0, diag, h1, l1, stage_T, ew, lane);
                oz_store_staged(p, m0, n0, il, cq + 32, 16, diag, h1, l1, stage_T, ew, lane);
            } else {
                oz_store_half(p, m0, n0, i, cq, diag, h0, l0);
                oz_store_half(p, m0, n0, i, cq + 32, diag, h1, l1);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(tmem, Cfg::TMEM_COLS);
}

template <class Cfg>
__global__ void __launch_bounds__(OZ_THREADS, Cfg::MIN_BLOCKS) ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                   const __grid_constant__ CUtensorMap tmB,
                                                                   const __grid_constant__ OzParams p) {
    oz_persistent<Cfg>(p.units, [&](int u, OzUnit& o) { oz_single_unit(&p, &tmA, &tmB, Cfg::ACC, u, o); });
}

// Grouped form: the tiles of every problem laid end to end; a unit finds its
// problem by binary search over the start offsets and reads that problem's
// tensor maps from global memory.  A tile is computed exactly as in the
// single-problem kernel.
template <class Cfg>
__global__ void __launch_bounds__(OZ_THREADS, 1) ozaki_gemm_grouped_kernel(const OzGroupDesc* __restrict__ d, int nd,
                                                                           int units) {
    oz_persistent<Cfg>(units, [&](int u, OzUnit& o) { oz_group_unit(d, nd, u, o); });
}

// Split K of the tail: the parts' level sums added in part order (the level-0
// parts are exact integers, so their sum is exact), then the epilogue of one
// element.  Block (tail tile, group of 8 tile rows) of 8 warps: warp w takes
// tile row 8 g + w and its lanes 32 consecutive columns at a time, so the
// workspace reads, the addend reads (at (i, j): tri addends are symmetric)
// and the row-direction stores are coalesced; the element arithmetic is
// oz_store_half's, so a split tile gives what an unsplit one would from the
// same level sums.
__device__ __forceinline__ void oz_tail_tile(const OzParams& p, int widx) {
    constexpr size_t tile_elems = (size_t)OZ_BM * OZ_BN;
    const int il = blockIdx.y * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    int tm, tn;
    oz_tile_coords(p, p.split_first + widx, tm, tn);
    const int i = tm * OZ_BM + il;
    if (i >= p.M) return;
    const bool diag = p.tri && tm == tn;
    const float sA = p.sa[i];
    const float2* base = p.ws + (size_t)widx * p.split_parts * tile_elems + (size_t)il * OZ_BN;
    for (int c0 = 0; c0 < OZ_BN; c0 += 32) {
        const int jl = c0 + lane, j = tn * OZ_BN + jl;
        if (j >= p.N || (diag && i > j)) continue;
        float hv = 0.f, lv = 0.f;
        for (int pp = 0; pp < p.split_parts; ++pp) {
            const float2 v = base[(size_t)pp * tile_elems + jl];
            hv += v.x;
            lv += v.y;
        }
        const float s = sA * p.sb[j];
        const float sh = hv + lv;
        const float bb = sh - hv;
        const float sl = (hv - (sh - bb)) + (lv - bb);
        const size_t off = (size_t)i * p.ldc + j;
        if (p.mode == OZ_OUT_PAIR) {
            p.Cp[off] = make_float2(sh * s, sl * s);
            continue;
        }
        double v = f2d_bits(sh * s) + f2d_bits(sl * s);
        if (p.alpha != 1.0) v *= p.alpha;
        if (p.D1) v += p.b1 * p.D1[off];
        if (p.D2) v += p.b2 * p.D2[off];
        if (p.D3) v += p.b3 * p.D3[off];
        p.Cd[off] = v;
        if (p.tri && i != j) p.Cd[(size_t)j * p.ldc + i] = v;
    }
}

__global__ void __launch_bounds__(256) oz_tail_kernel(const __grid_constant__ OzParams p) {
    oz_tail_tile(p, blockIdx.x);
}

// The tails of every split problem of a grouped launch: block x is split tile
// x - tail_start of the last problem whose tail_start <= x (problems without a
// split add no tiles, so that one is always a split problem).
__global__ void __launch_bounds__(256) oz_tail_grouped_kernel(const OzGroupDesc* __restrict__ d, int nd) {
    const int x = blockIdx.x;
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].tail_start <= x) lo = mid;
        else hi = mid - 1;
    }
    oz_tail_tile(d[lo].p, x - d[lo].tail_start);
}

// Accurate mode, second pass: C = alpha sum_c ws[c] + b1 D1 + b2 D2 (chunk order).
__global__ void __launch_bounds__(256) oz_chunk_reduce_kernel(const OzParams p) {
    const size_t total = (size_t)p.M * p.N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int c = 0; c < p.nchunks; ++c) v += p.wsd[(size_t)c * total + e];
        const size_t i = e / p.N, j = e - i * p.N;
        const size_t off = i * p.ldc + j;
        v *= p.alpha;
        if (p.D1) v += p.b1 * p.D1[off];
        if (p.D2) v += p.b2 * p.D2[off];
        p.Cd[off] = v;
    }
}

// ============================================================== host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static dme_status get_encoder() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return DME_ECUDA;
    }
    return DME_OK;
}

static dme_status make_slice_tmap(const SliceBuf& sb, int planes, CUtensorMap* out) {
    DME_TRY(get_encoder());
    cuuint64_t dims[3] = {(cuuint64_t)sb.Kp, (cuuint64_t)sb.rows, (cuuint64_t)sb.ns};
    cuuint64_t strides[2] = {(cuuint64_t)sb.Kp * 2, (cuuint64_t)sb.rows * sb.Kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)OZ_BM, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)sb.data, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return DME_ECUDA;
    }
    return DME_OK;
}

dme_status make_slice_tmaps(SliceBuf& sb) {
    if (sb.ns < 1 || sb.ns > 8) return set_error("slice buffer: 1 to 8 planes"), DME_EINVAL;
    DME_TRY(make_slice_tmap(sb, sb.ns, &sb.tmap));
    if (sb.ns > 4) DME_TRY(make_slice_tmap(sb, 4, &sb.tmap4));
    return DME_OK;
}

int slice_kpad(int k) { return (k + OZ_BK - 1) / OZ_BK * OZ_BK; }

size_t slice_buf_bytes(int rows, int k, int ns) { return (size_t)ns * rows * slice_kpad(k) * 2; }

dme_status oz_params(const SliceBuf& A, const SliceBuf& B, int cfg, OzParams* p) {
    if (cfg < 0 || cfg >= OZ_NCFG) return set_error("split gemm: unknown slice-pair configuration"), DME_EINVAL;
    if (A.ns < oz_cfg_slices_a(cfg) || B.ns < oz_cfg_slices_b(cfg) || A.scheme != oz_cfg_scheme(cfg) ||
        B.scheme != oz_cfg_scheme(cfg) || A.Kp != B.Kp)
        return set_error("split gemm: the slice buffers do not hold what the configuration reads"), DME_EINVAL;
    // a buffer with more planes than read is addressed through its four-plane map
    if ((A.ns > oz_cfg_slices_a(cfg) && oz_cfg_slices_a(cfg) != 4) ||
        (B.ns > oz_cfg_slices_b(cfg) && oz_cfg_slices_b(cfg) != 4))
        return set_error("split gemm: no tensor map spans the planes the configuration reads"), DME_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->M = A.rows;
    p->N = B.rows;
    p->Kp = A.Kp;
    p->cfg = cfg;
    p->sa = A.scale;
    p->sb = B.scale;
    p->alpha = 1.0;
    return DME_OK;
}

size_t oz_acc_ws_doubles(int M, int N, int K) {
    const int nk = slice_kpad(K) / OZ_BK;
    return (size_t)((nk + OZ_ACC_CHUNK_KB - 1) / OZ_ACC_CHUNK_KB) * M * N;
}

static int sm_count() {
    static const int nsm = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return std::max(c, 1);
    }();
    return nsm;
}

template <class Cfg>
static dme_status oz_launch_single(const CUtensorMap& tA, const CUtensorMap& tB, const OzParams& p, int grid,
                                   cudaStream_t st) {
    static const cudaError_t attr =
        cudaFuncSetAttribute(ozaki_gemm_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    DME_CUDA_TRY(attr);
    ozaki_gemm_kernel<Cfg><<<grid, OZ_THREADS, Cfg::SMEM, st>>>(tA, tB, p);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

// The split of K of a problem (not the accurate mode), from the problem alone: with a
// workspace (p.ws), the last partial wave in two K halves when it fills at most half
// of the SMs (it then takes about half a tile time instead of a whole one), or a
// single partial wave of skinny products in up to 4 K parts of at least 8 K blocks,
// within the SM count and the workspace's 2 x OZ_SPLIT_MAX_TAIL tile slots.  The
// single-problem and the grouped launches both apply it, so a problem gives the same
// bits in either.
static void oz_split_rule(OzParams& p, int nsm) {
    const int tiles = p.tiles;
    p.split_parts = 1;
    p.split_first = tiles;
    const int tail = tiles % nsm;
    if (p.ws && tiles > nsm && tail > 0 && tail <= OZ_SPLIT_MAX_TAIL && tail <= nsm / 2 && p.Kp / OZ_BK >= 16) {
        p.split_parts = 2;
        p.split_first = tiles - tail;
    } else if (p.ws && tiles <= nsm / 2 && tiles <= OZ_SPLIT_MAX_TAIL && p.Kp / OZ_BK >= 16) {
        int parts = 1;
        while (parts < 4 && tiles * (parts * 2) <= nsm && tiles * (parts * 2) <= 2 * OZ_SPLIT_MAX_TAIL &&
               p.Kp / OZ_BK / (parts * 2) >= 8)
            parts *= 2;
        if (parts > 1) {
            p.split_parts = parts;
            p.split_first = 0;
        }
    }
    p.units = p.split_first + (tiles - p.split_first) * p.split_parts;
}

dme_status launch_ozaki_gemm(const CUtensorMap& tA, const CUtensorMap& tB, OzParams p, cudaStream_t st) {
    if (p.M <= 0 || p.N <= 0) return DME_OK;
    if (p.Kp % OZ_BK != 0 || p.Kp > OZ_MAX_K) {
        set_error("ozaki gemm: K must be a multiple of 32 and at most 4096");
        return DME_EINVAL;
    }
    if (p.tri && p.M != p.N) {
        set_error("ozaki gemm: triangle mode needs M == N");
        return DME_EINVAL;
    }
    const bool acc = p.cfg == OZ_A21;
    if (acc && (p.mode != OZ_OUT_F64 || p.tri || p.D3 || !p.wsd)) {
        set_error("ozaki gemm: the accurate mode writes a full FP64 product through its chunk workspace");
        return DME_EINVAL;
    }
    const int nsm = sm_count();
    const int tmt = (p.M + OZ_BM - 1) / OZ_BM, tnt = (p.N + OZ_BN - 1) / OZ_BN;
    p.tiles_n = tnt;
    p.tiles = p.tri ? tnt * (tnt + 1) / 2 : tmt * tnt;
    const int tiles = p.tiles;
    p.split_parts = 1;
    p.split_first = tiles;
    p.nchunks = 1;
    if (acc) {
        p.nchunks = (p.Kp / OZ_BK + OZ_ACC_CHUNK_KB - 1) / OZ_ACC_CHUNK_KB;
        p.units = tiles * p.nchunks;
    } else {
        oz_split_rule(p, nsm);
    }
    // short and wide products (the Riccati update of large plans): two CTAs per SM (never
    // split: Kp / 32 < 16).  Narrower ones keep the four accumulators, so that a plan's
    // products round exactly as the grouped serving kernel's.
    const bool shortk = !acc && p.Kp <= 2 * OZ_BK && tiles > nsm;
    const int grid = std::min(p.units, shortk ? 2 * nsm : nsm);
    switch (p.cfg) {
        case OZ_P10:
            DME_TRY(shortk ? oz_launch_single<CfgP10s>(tA, tB, p, grid, st) : oz_launch_single<CfgP10>(tA, tB, p, grid, st));
            break;
        case OZ_P13:
            DME_TRY(shortk ? oz_launch_single<CfgP13s>(tA, tB, p, grid, st) : oz_launch_single<CfgP13>(tA, tB, p, grid, st));
            break;
        case OZ_P14:
            if (shortk) DME_TRY(oz_launch_single<CfgP14s>(tA, tB, p, grid, st));
            else if (p.units <= nsm) DME_TRY(oz_launch_single<CfgP14e>(tA, tB, p, grid, st));
            else DME_TRY(oz_launch_single<CfgP14>(tA, tB, p, grid, st));
            break;
        case OZ_A21: DME_TRY(oz_launch_single<CfgA21>(tA, tB, p, grid, st)); break;
        default: return set_error("ozaki gemm: unknown configuration"), DME_EINVAL;
    }
    if (p.split_parts > 1) {
        oz_tail_kernel<<<dim3(tiles - p.split_first, OZ_BM / 8), 256, 0, st>>>(p);
        DME_CUDA_TRY(cudaGetLastError());
    }
    if (acc) {
        const size_t total = (size_t)p.M * p.N;
        const int g = (int)std::min<size_t>((total + 255) / 256, (size_t)nsm * 8);
        oz_chunk_reduce_kernel<<<g, 256, 0, st>>>(p);
        DME_CUDA_TRY(cudaGetLastError());
    }
    return DME_OK;
}

template <class Cfg>
static dme_status oz_grouped_attr() {
    static const cudaError_t attr =
        cudaFuncSetAttribute(ozaki_gemm_grouped_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
    DME_CUDA_TRY(attr);
    return DME_OK;
}

dme_status ozaki_grouped_prepare() {
    DME_TRY(oz_grouped_attr<CfgP13>());
    DME_TRY(oz_grouped_attr<CfgP14e>());
    return DME_OK;
}

dme_status launch_ozaki_grouped(std::vector<OzGroupDesc>& items, OzGroupDesc* dev_desc, cudaStream_t st,
                                DescArena* arena) {
    // configurations of one launch: 10 and 13 products (4 x 4 slices, the 13-product
    // kernel cutting the 10-product problems at level 3), or 14 alone
    int total = 0, cfg = -1;
    std::vector<OzGroupDesc> live;
    for (auto& it : items) {
        OzParams& p = it.p;
        if (p.M <= 0 || p.N <= 0) continue;
        const int cls = p.cfg == OZ_P10 ? OZ_P13 : p.cfg;
        if (p.Kp % OZ_BK != 0 || p.Kp > OZ_MAX_K || (p.tri && p.M != p.N) || p.cfg == OZ_A21 ||
            (cfg >= 0 && cls != cfg)) {
            set_error("ozaki grouped gemm: bad problem shape or mixed configurations");
            return DME_EINVAL;
        }
        cfg = cls;
        const int tmt = (p.M + OZ_BM - 1) / OZ_BM, tnt = (p.N + OZ_BN - 1) / OZ_BN;
        p.tiles_n = tnt;
        p.tiles = p.tri ? tnt * (tnt + 1) / 2 : tmt * tnt;
        oz_split_rule(p, sm_count());
        live.push_back(it);
    }
    // the longest units (K per unit) first, so that they start in the first wave
    std::stable_sort(live.begin(), live.end(), [](const OzGroupDesc& x, const OzGroupDesc& y) {
        return x.p.Kp / x.p.split_parts > y.p.Kp / y.p.split_parts;
    });
    int tail_total = 0;
    for (auto& it : live) {
        it.start = total;
        total += it.p.units;
        it.tail_start = tail_total;
        if (it.p.split_parts > 1) tail_total += it.p.tiles - it.p.split_first;
    }
    if (total == 0) return DME_OK;
    DME_TRY(ozaki_grouped_prepare());
    OzGroupDesc* d = dev_desc;
    if (arena) {
        d = static_cast<OzGroupDesc*>(arena->put(live.data(), live.size() * sizeof(OzGroupDesc)));
        if (!d) return set_error("ozaki grouped gemm: descriptor arena full"), DME_ENOMEM;
    } else {
        DME_CUDA_TRY(cudaMemcpyAsync(d, live.data(), live.size() * sizeof(OzGroupDesc), cudaMemcpyHostToDevice, st));
    }
    const int grid = std::min(total, sm_count());
    const int nd = (int)live.size();
    switch (cfg) {
        case OZ_P13:
            ozaki_gemm_grouped_kernel<CfgP13><<<grid, OZ_THREADS, CfgP13::SMEM, st>>>(d, nd, total);
            break;
        default:   // serving problems are small: the staged two-stage form of 14 products
            ozaki_gemm_grouped_kernel<CfgP14e><<<grid, OZ_THREADS, CfgP14e::SMEM, st>>>(d, nd, total);
            break;
    }
    DME_CUDA_TRY(cudaGetLastError());
    // the parts of the split problems added and their epilogues run, in one launch
    if (tail_total > 0) {
        oz_tail_grouped_kernel<<<dim3(tail_total, OZ_BM / 8), 256, 0, st>>>(d, nd);
        DME_CUDA_TRY(cudaGetLastError());
    }
    return DME_OK;
}

}  // namespace dme

// ============================================================== allocation-free split GEMM
// dme_gemm_split_noalloc keeps its scratch (the bf16 slices of A and B, their
// row scales and a status word) in this file-scope device array instead of
// allocating it.  Every device that loads the library holds the array until
// the process exits; every call shares it.
namespace dme {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;    // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];

// Device address of the scratch array on the current device.  The first call
// on a device looks it up (with that device current) and caches it.
static dme_status noalloc_scratch_address(void** out) {
    int dev = 0;
    DME_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error("device ordinal out of range"), DME_EINVAL;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return DME_ECUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return DME_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace dme

extern "C" dme_status dme_gemm_split_noalloc(int M, int N, int K, const double* A, const double* B, double* C,
                                             void* cuda_stream) {
    using namespace dme;
    if (M < 0 || N < 0 || K < 1 || K > OZ_MAX_K || !A || !B || !C)
        return set_error("dme_gemm_split_noalloc: need 1 <= K <= 4096 and non-null A, B, C"), DME_EINVAL;
    if (M == 0 || N == 0) return DME_OK;
    try {
        const int Kp = slice_kpad(K);
        // scratch layout: status | scales of A | scales of B | slices of A | slices of B
        const size_t off_sa = 256;
        const size_t off_sb = off_sa + align256(sizeof(float) * (size_t)M);
        const size_t off_a = off_sb + align256(sizeof(float) * (size_t)N);
        const size_t off_b = off_a + align256(slice_buf_bytes(M, K, OZ_SLICES_FIXED));
        const size_t need = off_b + align256(slice_buf_bytes(N, K, OZ_SLICES_STEP));
        if (need > kNoAllocScratchBytes) {
            set_error("dme_gemm_split_noalloc: M=" + std::to_string(M) + " N=" + std::to_string(N) +
                      " K=" + std::to_string(K) + " needs " + std::to_string(need) +
                      " bytes of scratch, more than its 8 MiB ((5 M + 4 N) * roundup(K, 32) * 2 bytes of slices"
                      " plus row scales)");
            return DME_EINVAL;
        }
        unsigned char* base = nullptr;
        DME_TRY(noalloc_scratch_address(reinterpret_cast<void**>(&base)));
        cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
        int* status = reinterpret_cast<int*>(base);
        SliceBuf sa, sb;
        sa.rows = M;
        sa.k = K;
        sa.Kp = Kp;
        sa.ns = OZ_SLICES_FIXED;
        sa.scale = reinterpret_cast<float*>(base + off_sa);
        sa.data = reinterpret_cast<__nv_bfloat16*>(base + off_a);
        sb.rows = N;
        sb.k = K;
        sb.Kp = Kp;
        sb.ns = OZ_SLICES_STEP;
        sb.scale = reinterpret_cast<float*>(base + off_sb);
        sb.data = reinterpret_cast<__nv_bfloat16*>(base + off_b);
        DME_TRY(make_slice_tmaps(sa));
        DME_TRY(make_slice_tmaps(sb));
        // the array keeps the previous call's contents: the status word must start at zero
        // (slices, padding and scales are rewritten in full below)
        DME_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
        launch_slice_rows_f64(A, M, K, K, sa, st);
        launch_slice_rows_f64(B, N, K, K, sb, st);
        OzParams o;
        DME_TRY(oz_params(sa, sb, OZ_P14, &o));
        o.mode = OZ_OUT_F64;
        o.ldc = N;
        o.Cd = C;
        o.status = status;
        DME_TRY(launch_ozaki_gemm(oz_tmap_a(sa, OZ_P14), oz_tmap_b(sb, OZ_P14), o, st));
        int hs = 0;
        DME_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        DME_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs) {
            set_error("dme_gemm_split_noalloc: device status " + std::to_string(hs));
            return DME_ECUDA;
        }
        return DME_OK;
    } catch (...) {
        set_error("dme_gemm_split_noalloc: internal error");
        return DME_EINVAL;
    }
}
