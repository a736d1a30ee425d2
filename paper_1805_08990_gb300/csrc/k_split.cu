// Split-precision congruence G P G^T on tcgen05 tensor cores.
//
// Error-free slicing (after Ozaki, Ogita, Oishi & Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication", Numer. Algorithms 59, 2012): each row r of an operand is
// scaled by sigma_r = 2^E_r > max |x_r.| and cut into bf16 slices
//     x / sigma = d0 2^-6 + d1 2^-13 + d2 2^-20 + d3 2^-27 + d4 2^-34 + res,
// with integers |d_t| <= 64.  The fixed operand (G = E^T or S, the A side)
// keeps five slices (|res| <= 2^-35): its slicing error is the same at every
// step and would otherwise add up coherently over the horizon.  The per-step
// operand (P or U, the B side) keeps four (|res| <= 2^-28); its errors are
// fresh each step and averaged by the congruence.
// A slice product d_s d_t 2^-(12+7(s+t)) is exact in bf16 x bf16, and a level
// l = s + t sums K <= 4096 such products: at most 2^24 units of
// 2^-(12+7l), so the fp32 tensor-core accumulation of level 0 is exact
// whatever its rounding mode, and the other levels round far below the
// slice residuals.  The 14 pairs with s + t <= 4 are accumulated in four TMEM
// accumulators (levels 0, 1, 2 and 3+4); the epilogue adds them as a
// two-float (hi = level 0, exact; lo = levels 1-4) and scales by
// sigma_A,i sigma_B,j.
//
// Kernel shape: one CTA per 128 x 128 output tile, 10 warps:
//   warp 0  TMA producer (one thread): 3-stage ring, each stage holds the 5
//           slices of a 128 x 32 A tile and the 4 slices of a 128 x 32 B tile
//           (72 KB, 64-byte swizzled rows),
//   warp 1  TMEM allocator + MMA issuer (one thread): 28 tcgen05.mma per stage,
//   warps 2-9 epilogue: tcgen05.ld of the 4 accumulators (512 TMEM columns),
//           two warps per TMEM lane quadrant, each on half of the tile's columns.
// Both operands are K-major (row-major with K contiguous):
//   C[i][j] = sum_k A[i][k] B[j][k].
#include "dme_internal.h"
#include "split_internal.h"
#include "tc_ptx.cuh"

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace dme {

using namespace tc;

constexpr int OZ_BM = 128, OZ_BN = 128, OZ_BK = 32, OZ_STAGES = 3;
constexpr int OZ_SLICE_BYTES = OZ_BM * OZ_BK * 2;                 // 8 KB per slice tile
constexpr int OZ_A_BYTES = OZ_SLICES_A * OZ_SLICE_BYTES;         // 40 KB per stage
constexpr int OZ_B_BYTES = OZ_SLICES_B * OZ_SLICE_BYTES;         // 32 KB per stage
constexpr int OZ_STAGE_BYTES = OZ_A_BYTES + OZ_B_BYTES;          // 72 KB
constexpr int OZ_SMEM_BYTES = OZ_STAGES * OZ_STAGE_BYTES + 1024 + 256;
constexpr int OZ_MAX_LEVEL = 4;                                   // pairs with s + t <= 4
constexpr int OZ_NACC = 4;                                        // accumulators: levels 0, 1, 2, 3+4
constexpr uint64_t OZ_TIMEOUT_NS = 2000000000ull;             // 2 s per wait
constexpr int OZ_EPI_WARPS = 8;                                  // two per TMEM lane quadrant
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;               // producer + MMA warps + epilogue
constexpr int OZ_EPI_COLS = OZ_BN / (OZ_EPI_WARPS / 4);          // columns per epilogue warp
constexpr uint32_t OZ_IDESC = idesc_bf16_f32(OZ_BM, OZ_BN);

// ============================================================== slicing
__device__ __forceinline__ long long round_shift(unsigned long long mag, int shift) {
    if (shift >= 64) return 0;
    if (shift <= 0) return (long long)(mag << (-shift));
    return (long long)((mag + (1ull << (shift - 1))) >> shift);
}

// round(x * 2^(41 - E)) for a double x (|x| < 2^E, so |result| <= 2^41)
__device__ __forceinline__ long long fixed41_d(double x, int E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF) return 0;
    const unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const long long v = round_shift(M, 1075 + E - 41 - ex);
    return (b >> 63) ? -v : v;
}

// round(f * 2^(41 - E)) for a float f
__device__ __forceinline__ long long fixed41_f(float f, int E) {
    const unsigned int b = __float_as_uint(f);
    const int ef = (int)((b >> 23) & 0xFF);
    if (ef == 0 || ef == 0xFF) return 0;
    const unsigned long long M = (b & 0x7FFFFFu) | 0x800000u;
    const long long v = round_shift(M, 109 + E - ef);
    return (b >> 31) ? -v : v;
}

// The NS base-2^7 digits of V (|V| < 2^41) with round-to-nearest,
// d_t = round(r_t / 2^(35-7t)), r_{t+1} = r_t - d_t 2^(35-7t), in 32-bit
// arithmetic: V = h 2^21 + l with 0 <= l < 2^21; digits 0 and 1 come from h
// alone (l < 2^21 cannot change those floors), digit 2 is h plus the rounding
// carry of l, and digits 3 and 4 come from the remainder l - carry 2^21.
template <int NS>
__device__ __forceinline__ void digits7(long long V, int (&dg)[5]) {
    int h = (int)(V >> 21);
    const int l = (int)(V - ((long long)h << 21));
    int d = (h + (1 << 13)) >> 14;
    h -= d << 14;
    dg[0] = d;
    d = (h + (1 << 6)) >> 7;
    h -= d << 7;
    dg[1] = d;
    const int c = l >= (1 << 20) ? 1 : 0;
    dg[2] = h + c;
    int r = l - (c << 21);
    d = (r + (1 << 13)) >> 14;
    r -= d << 14;
    dg[3] = d;
    dg[4] = (r + (1 << 6)) >> 7;
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

// One warp per row: pass 1 finds the row's max exponent, pass 2 writes the
// NS slices (zero beyond `cols`, up to Kp) and the row scale 2^E.  The value
// is first rounded to a 41-bit fixed-point integer V = round(x 2^(41-E)); the
// slices are the base-2^7 digits of V with round-to-nearest:
// d_t = round(r_t / 2^(35-7t)), r_{t+1} = r_t - d_t 2^(35-7t).
// Each lane handles 4 consecutive entries (32-byte loads, 8-byte stores per plane).
template <bool PAIR, int NS>
__device__ __forceinline__ void slice_row_warp(const double* __restrict__ X, const float2* __restrict__ Xp, int row,
                                               int cols, int ldx, __nv_bfloat16* __restrict__ out, int Kp,
                                               float* __restrict__ scale, int prow) {
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)row * ldx;
    const bool vec = (ldx % 2) == 0;
    double d[4];
    float2 f[4];
    // pass 1: largest magnitude (as exponent)
    int emax = -100000;
    for (int k = 4 * lane; k < cols; k += 128) {
        load4<PAIR>(X, Xp, base, k, cols, vec, d, f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int e;
            if (PAIR) {
                const unsigned int b = __float_as_uint(f[u].x) & 0x7FFFFFFFu;
                const int ef = (int)(b >> 23);
                e = (b == 0 || ef == 0) ? -100000 : ef - 127;
            } else {
                const unsigned long long b = (unsigned long long)__double_as_longlong(d[u]);
                const int ed = (int)((b >> 52) & 0x7FF);
                e = (ed == 0) ? -100000 : ed - 1023;
            }
            emax = max(emax, e);
        }
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
            for (int u = 0; u < 4; ++u)
                V[u] = PAIR ? fixed41_f(f[u].x, E) + fixed41_f(f[u].y, E) : fixed41_d(d[u], E);
        }
        const size_t o = (size_t)row * Kp + k;
        int dg[4][5];
#pragma unroll
        for (int u = 0; u < 4; ++u) digits7<NS>(V[u], dg[u]);
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            const float unit = __int_as_float((127 - 6 - 7 * t) << 23);     // 2^(-6-7t), exact
            float q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) q[u] = (float)dg[u][t] * unit;      // |d| <= 64: exact in float
            const __nv_bfloat162 p01 = __floats2bfloat162_rn(q[0], q[1]);
            const __nv_bfloat162 p23 = __floats2bfloat162_rn(q[2], q[3]);
            uint2 w;
            w.x = *reinterpret_cast<const unsigned int*>(&p01);
            w.y = *reinterpret_cast<const unsigned int*>(&p23);
            *reinterpret_cast<uint2*>(out + t * plane + o) = w;
        }
    }
}

template <bool PAIR, int NS>
__global__ void __launch_bounds__(256) slice_rows_kernel(const double* __restrict__ X, const float2* __restrict__ Xp,
                                                         int rows, int cols, int ldx, __nv_bfloat16* __restrict__ out,
                                                         int Kp, float* __restrict__ scale, int prow) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (row >= rows) return;
    slice_row_warp<PAIR, NS>(X, Xp, row, cols, ldx, out, Kp, scale, prow);
}

// Grouped slicing (serving): the rows of several problems laid end to end,
// a warp per row; warp w finds its problem by a binary search over row0.
template <bool PAIR, int NS>
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
    slice_row_warp<PAIR, NS>(q.X, q.Xp, g - q.row0, q.cols, q.ldx, q.out, q.Kp, q.scale, q.prow);
}

// Long rows (Kp > 1024): one CTA of 256 threads per row; each thread keeps G
// groups of 4 consecutive entries (k = 4 tid + 1024 g) in registers, so the
// row is read from memory once; the row maximum is a block reduction.  Same
// digits as slice_rows_kernel.
template <bool PAIR, int NS, int G>
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
        for (int u = 0; u < 4; ++u) {
            int e;
            if (PAIR) {
                const unsigned int b = __float_as_uint(f[g][u].x) & 0x7FFFFFFFu;
                const int ef = (int)(b >> 23);
                e = (b == 0 || ef == 0) ? -100000 : ef - 127;
            } else {
                const unsigned long long b = (unsigned long long)__double_as_longlong(d[g][u]);
                const int ed = (int)((b >> 52) & 0x7FF);
                e = (ed == 0) ? -100000 : ed - 1023;
            }
            emax = max(emax, e);
        }
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
            for (int u = 0; u < 4; ++u)
                V[u] = PAIR ? fixed41_f(f[g][u].x, E) + fixed41_f(f[g][u].y, E) : fixed41_d(d[g][u], E);
        }
        const size_t o = (size_t)row * Kp + k;
        int dg[4][5];
#pragma unroll
        for (int u = 0; u < 4; ++u) digits7<NS>(V[u], dg[u]);
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            const float unit = __int_as_float((127 - 6 - 7 * t) << 23);
            float q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) q[u] = (float)dg[u][t] * unit;
            const __nv_bfloat162 p01 = __floats2bfloat162_rn(q[0], q[1]);
            const __nv_bfloat162 p23 = __floats2bfloat162_rn(q[2], q[3]);
            uint2 w;
            w.x = *reinterpret_cast<const unsigned int*>(&p01);
            w.y = *reinterpret_cast<const unsigned int*>(&p23);
            *reinterpret_cast<uint2*>(out + t * plane + o) = w;
        }
    }
}

template <bool PAIR, int NS>
static void slice_launch(const double* X, const float2* Xp, int rows, int cols, int ldx, const SliceBuf& sb,
                         cudaStream_t st) {
    if (rows <= 0 || rows > sb.rows) return;
    const int pr = sb.rows;
    if (sb.Kp > 2048)
        slice_long_rows_kernel<PAIR, NS, 4><<<rows, 256, 0, st>>>(X, Xp, rows, cols, ldx, sb.data, sb.Kp, sb.scale, pr);
    else if (sb.Kp > 1024)
        slice_long_rows_kernel<PAIR, NS, 2><<<rows, 256, 0, st>>>(X, Xp, rows, cols, ldx, sb.data, sb.Kp, sb.scale, pr);
    else
        slice_rows_kernel<PAIR, NS><<<(rows + 7) / 8, 256, 0, st>>>(X, Xp, rows, cols, ldx, sb.data, sb.Kp, sb.scale,
                                                                     pr);
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
    if (pair) slice_rows_grouped_kernel<true, 4><<<grid, 256, 0, st>>>(dd, (int)items.size(), total);
    else slice_rows_grouped_kernel<false, 4><<<grid, 256, 0, st>>>(dd, (int)items.size(), total);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

void launch_slice_rows_f64(const double* X, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st) {
    if (sb.ns == 5) slice_launch<false, 5>(X, nullptr, rows, cols, ldx, sb, st);
    else slice_launch<false, 4>(X, nullptr, rows, cols, ldx, sb, st);
}

void launch_slice_rows_pair(const float2* Xp, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st) {
    if (sb.ns == 5) slice_launch<true, 5>(nullptr, Xp, rows, cols, ldx, sb, st);
    else slice_launch<true, 4>(nullptr, Xp, rows, cols, ldx, sb, st);
}

// ============================================================== tcgen05 GEMM
// Tile order.  Rectangular grids run in groups of OZ_GROUP tile rows, column
// by column inside a group, so the CTAs resident at one time touch about
// OZ_GROUP row tiles of A and 152/OZ_GROUP column tiles of B, which stay in L2.
// Triangle grids enumerate (tm <= tn) row by row.
constexpr int OZ_GROUP = 8;

__device__ __forceinline__ void oz_tile_coords(const OzParams& p, int t, int& tm, int& tn) {
    if (p.tri) {
        int T = p.tiles_n, r = 0, rem = t;
        while (rem >= T - r) {
            rem -= T - r;
            ++r;
        }
        tm = r;
        tn = r + rem;
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

// One 128 x 128 output tile (index t of problem p) by one CTA; tmA / tmB are
// the addresses of the tensor maps (kernel parameters or global memory).
__device__ __forceinline__ void oz_gemm_tile(const CUtensorMap* tmA, const CUtensorMap* tmB, const OzParams& p,
                                             int t, int part, int nparts, int widx) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OZ_STAGES * OZ_STAGE_BYTES);
    // bars[0..S): full, bars[S..2S): empty, bars[2S]: accumulators ready
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * OZ_STAGES + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tm, tn;
    oz_tile_coords(p, t, tm, tn);
    const int m0 = tm * OZ_BM, n0 = tn * OZ_BN;
    const int nk_all = p.Kp / OZ_BK;
    const int kb0 = part * nk_all / nparts;                 // this CTA's K blocks [kb0, kb0 + nk)
    const int nk = (part + 1) * nk_all / nparts - kb0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[OZ_STAGES + s]), 1);
        }
        mbar_init(smem_u32(&bars[2 * OZ_STAGES]), 1);
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        tma_prefetch_desc(tmA);
        tma_prefetch_desc(tmB);
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), 512);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued[OZ_STAGES] = {0, 0, 0};
            bool ok = true;
            for (int it = 0; it < nk && ok; ++it) {
                const int kb = kb0 + it;
                const int s = it % OZ_STAGES;
                const uint32_t ph = (it / OZ_STAGES) & 1;
                if (it >= OZ_STAGES && !mbar_wait(smem_u32(&bars[OZ_STAGES + s]), ph ^ 1, OZ_TIMEOUT_NS)) {
                    ok = false;
                    break;
                }
                const uint32_t full = smem_u32(&bars[s]);
                uint8_t* st = smem + s * OZ_STAGE_BYTES;
                mbar_arrive_expect_tx(full, OZ_STAGE_BYTES);
                tma_load_3d(smem_u32(st), tmA, full, kb * OZ_BK, m0, 0);
                tma_load_3d(smem_u32(st + OZ_A_BYTES), tmB, full, kb * OZ_BK, n0, 0);
                issued[s]++;
                // spread over the K loop: pull the epilogue's addend rows (full 128-column
                // segments only, all in bounds) into L2, one row per k block
                const int pr = it * nparts + part;
                if (p.mode == OZ_OUT_F64 && pr < OZ_BM && m0 + pr < p.M && n0 + OZ_BN <= p.N &&
                    (p.ldc % 2) == 0) {
                    const size_t off = (size_t)(m0 + pr) * p.ldc + n0;
                    // the bulk prefetch needs a 16-byte aligned start (addends may be caller memory)
                    if (p.D1 && ((reinterpret_cast<uintptr_t>(p.D1 + off) & 15) == 0))
                        prefetch_l2_bulk(p.D1 + off, OZ_BN * sizeof(double));
                    if (p.D2 && ((reinterpret_cast<uintptr_t>(p.D2 + off) & 15) == 0))
                        prefetch_l2_bulk(p.D2 + off, OZ_BN * sizeof(double));
                }
            }
            if (!ok) atomicOr(p.status, DEV_TIMEOUT);
            // every load this thread issued has landed before the CTA may exit
            for (int s = 0; s < OZ_STAGES; ++s)
                if (issued[s] > 0 && !mbar_wait(smem_u32(&bars[s]), (issued[s] - 1) & 1, OZ_TIMEOUT_NS))
                    atomicOr(p.status, DEV_TIMEOUT);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int it = 0; it < nk; ++it) {
                const int s = it % OZ_STAGES;
                const uint32_t ph = (it / OZ_STAGES) & 1;
                if (!mbar_wait(smem_u32(&bars[s]), ph, OZ_TIMEOUT_NS)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t a0 = smem_u32(smem + s * OZ_STAGE_BYTES);
                const uint32_t b0 = a0 + OZ_A_BYTES;
#pragma unroll
                for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
                    for (int sa = 0; sa < OZ_SLICES_A; ++sa) {
#pragma unroll
                        for (int sb = 0; sb < OZ_SLICES_B; ++sb) {
                            if (sa + sb > OZ_MAX_LEVEL) continue;
                            const int lvl = (sa + sb < OZ_NACC - 1) ? sa + sb : OZ_NACC - 1;
                            const uint64_t ad = desc_kmajor_sw64(a0 + sa * OZ_SLICE_BYTES + kk * 32);
                            const uint64_t bd = desc_kmajor_sw64(b0 + sb * OZ_SLICE_BYTES + kk * 32);
                            // the pairs (0, t) come first for every accumulator t: at the very
                            // first k step they overwrite it, everything else accumulates
                            const uint32_t acc = (it == 0 && kk == 0 && sa == 0) ? 0u : 1u;
                            mma_bf16(tmem + (uint32_t)(lvl * OZ_BN), ad, bd, OZ_IDESC, acc);
                        }
                    }
                }
                mma_commit(smem_u32(&bars[OZ_STAGES + s]));
            }
            if (!ok) atomicOr(p.status, DEV_TIMEOUT);
            mma_commit(smem_u32(&bars[2 * OZ_STAGES]));
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = tile rows, columns
        // [cq, cq + OZ_EPI_COLS) with cq = OZ_EPI_COLS * ((w - 2) / 4)
        const int q = warp & 3;
        const int ew = warp - 2;                                   // 0 .. OZ_EPI_WARPS-1
        const int cq = OZ_EPI_COLS * (ew / 4);
        const int i = m0 + 32 * q + lane;
        const bool ready_here = mbar_wait(smem_u32(&bars[2 * OZ_STAGES]), 0, OZ_TIMEOUT_NS);
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
        const bool ready = all_ready != 0;
        fence_after_sync();
        if (!ready) {
            if (lane == 0) atomicOr(p.status, DEV_TIMEOUT);
        } else {
            const int il = 32 * q + lane;                          // tile row of this thread
            const size_t tile_elems = (size_t)OZ_BM * OZ_BN;
            // level sums of 32 columns starting at c * 32: hi = level 0 (exact), lo = levels 1-4
            auto tmem_chunk = [&](int c, float (&hv)[32], float (&lv)[32]) {
                uint32_t r0[32], r1[32], r2[32], r3[32];
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c * 32);
                tmem_ld_32x32b_x32(ta, r0);
                tmem_ld_32x32b_x32(ta + OZ_BN, r1);
                tmem_ld_32x32b_x32(ta + 2 * OZ_BN, r2);
                tmem_ld_32x32b_x32(ta + 3 * OZ_BN, r3);
                tmem_ld_wait();
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    hv[jj] = __uint_as_float(r0[jj]);
                    lv[jj] = (__uint_as_float(r1[jj]) + __uint_as_float(r2[jj])) + __uint_as_float(r3[jj]);
                }
            };
            bool run_epilogue = true;
            if (nparts > 1) {
                // split K: publish this part's sums, count arrivals; the last part finishes
                float2* mine = p.ws + ((size_t)widx * nparts + part) * tile_elems;
#pragma unroll 1
                for (int c = cq / 32; c < (cq + OZ_EPI_COLS) / 32; ++c) {
                    float hv[32], lv[32];
                    tmem_chunk(c, hv, lv);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) mine[(size_t)il * OZ_BN + c * 32 + jj] = make_float2(hv[jj], lv[jj]);
                }
                __threadfence();
                asm volatile("bar.sync 1, 256;" ::: "memory");
                volatile int* flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
                if (ew == 0 && lane == 0) *flag = atomicAdd(p.ws_cnt + widx, 1);
                asm volatile("bar.sync 1, 256;" ::: "memory");
                run_epilogue = (*flag == nparts - 1);
                if (run_epilogue) {
                    __threadfence();
                    if (ew == 0 && lane == 0) p.ws_cnt[widx] = 0;    // ready for the next launch
                }
            }
            // level sums of a chunk: from TMEM, or the parts' sums added in part order
            auto chunk = [&](int c, float (&hv)[32], float (&lv)[32]) {
                if (nparts == 1) {
                    tmem_chunk(c, hv, lv);
                    return;
                }
                const float2* base = p.ws + (size_t)widx * nparts * tile_elems + (size_t)il * OZ_BN + c * 32;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    hv[jj] = 0.0f;
                    lv[jj] = 0.0f;
                }
                for (int pp = 0; pp < nparts; ++pp) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const float2 v = base[pp * tile_elems + jj];
                        hv[jj] += v.x;
                        lv[jj] += v.y;
                    }
                }
            };
            if (run_epilogue && p.mode == OZ_OUT_PAIR) {
                const float sA = (i < p.M) ? p.sa[i] : 0.0f;
#pragma unroll 1
                for (int c = cq / 32; c < (cq + OZ_EPI_COLS) / 32; ++c) {
                    float hv[32], lv[32];
                    chunk(c, hv, lv);
                    if (i >= p.M) continue;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const int j = n0 + c * 32 + jj;
                        if (j >= p.N) break;
                        const float s = sA * p.sb[j];
                        // TwoSum: (sh, sl) = hi + lo exactly
                        const float sh = hv[jj] + lv[jj];
                        const float bb = sh - hv[jj];
                        const float sl = (hv[jj] - (sh - bb)) + (lv[jj] - bb);
                        p.Cp[(size_t)i * p.ldc + j] = make_float2(sh * s, sl * s);
                    }
                }
            } else if (run_epilogue) {
                // FP64 output, staged through shared memory (the operand stages are idle now: every
                // MMA has completed, so every TMA load they consumed has landed):
                // (1) each thread converts its row segment of the tile into T[row][col];
                // (2) the epilogue warps write row segments of C coalesced, adding the addends;
                // (3) for a symmetric output they write the mirror from T's columns, coalesced.
                constexpr int TLD = OZ_BN + 1;
                double* T = reinterpret_cast<double*>(smem);
                const float sA = (i < p.M) ? p.sa[i] : 0.0f;
#pragma unroll 1
                for (int c = cq / 32; c < (cq + OZ_EPI_COLS) / 32; ++c) {
                    float hv[32], lv[32];
                    chunk(c, hv, lv);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const int j = n0 + c * 32 + jj;
                        const float s = (j < p.N) ? sA * p.sb[j] : 0.0f;
                        const float sh = hv[jj] + lv[jj];
                        const float bb = sh - hv[jj];
                        const float sl = (hv[jj] - (sh - bb)) + (lv[jj] - bb);
                        T[il * TLD + c * 32 + jj] = f2d_bits(sh * s) + f2d_bits(sl * s);
                    }
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");
                const double alpha = p.alpha;
                // rows ew, ew+8, ..., in batches of 4 rows x 4 column groups (the whole tile width):
                // 16 independent addend loads in flight per thread
                for (int rb = 0; rb < OZ_BM / OZ_EPI_WARPS; rb += 4) {
                    double a1[4][OZ_BN / 32], a2[4][OZ_BN / 32];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int gi = m0 + ew + OZ_EPI_WARPS * (rb + u);
#pragma unroll
                        for (int h = 0; h < OZ_BN / 32; ++h) {
                            const int gj = n0 + lane + 32 * h;
                            const bool in = gi < p.M && gj < p.N;
                            const size_t off = (size_t)gi * p.ldc + gj;
                            a1[u][h] = (in && p.D1) ? p.D1[off] : 0.0;
                            a2[u][h] = (in && p.D2) ? p.D2[off] : 0.0;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int r = ew + OZ_EPI_WARPS * (rb + u);
                        const int gi = m0 + r;
                        if (gi >= p.M) continue;
#pragma unroll
                        for (int h = 0; h < OZ_BN / 32; ++h) {
                            const int cc = lane + 32 * h;
                            const int gj = n0 + cc;
                            if (gj >= p.N || (p.tri && gi > gj)) continue;
                            const size_t off = (size_t)gi * p.ldc + gj;
                            double v = T[r * TLD + cc];
                            if (alpha != 1.0) v *= alpha;
                            if (p.D1) v += p.b1 * a1[u][h];
                            if (p.D2) v += p.b2 * a2[u][h];
                            if (p.D3) v += p.b3 * p.D3[off];
                            p.Cd[off] = v;
                            T[r * TLD + cc] = v;
                        }
                    }
                }
                if (p.tri) {
                    asm volatile("bar.sync 1, 256;" ::: "memory");
                    for (int cc = ew; cc < OZ_BN; cc += OZ_EPI_WARPS) {
                        const int gj = n0 + cc;
                        if (gj >= p.N) continue;
#pragma unroll
                        for (int h = 0; h < OZ_BM / 32; ++h) {
                            const int r = lane + 32 * h;
                            const int gi = m0 + r;
                            if (gi >= p.M || gi >= gj) continue;
                            p.Cd[(size_t)gj * p.ldc + gi] = T[r * TLD + cc];
                        }
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(tmem, 512);
}

__global__ void __launch_bounds__(OZ_THREADS, 1) ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                             const __grid_constant__ CUtensorMap tmB,
                                                             const OzParams p) {
    const int b = blockIdx.x;
    if (p.split_parts <= 1 || b < p.split_first) {
        oz_gemm_tile(&tmA, &tmB, p, b, 0, 1, 0);
    } else {
        const int j = b - p.split_first;
        oz_gemm_tile(&tmA, &tmB, p, p.split_first + j / p.split_parts, j % p.split_parts, p.split_parts,
                     j / p.split_parts);
    }
}

// Grouped form: the tiles of every problem laid end to end; a CTA finds its
// problem by binary search over the start offsets and reads that problem's
// tensor maps from global memory.  A tile is computed exactly as in the
// single-problem kernel.
__global__ void __launch_bounds__(OZ_THREADS, 1) ozaki_gemm_grouped_kernel(const OzGroupDesc* __restrict__ d, int nd) {
    const int b = blockIdx.x;
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].start <= b) lo = mid;
        else hi = mid - 1;
    }
    oz_gemm_tile(&d[lo].tmA, &d[lo].tmB, d[lo].p, b - d[lo].start, 0, 1, 0);
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

dme_status make_slice_tmap(const SliceBuf& sb, CUtensorMap* out) {
    DME_TRY(get_encoder());
    cuuint64_t dims[3] = {(cuuint64_t)sb.Kp, (cuuint64_t)sb.rows, (cuuint64_t)sb.ns};
    cuuint64_t strides[2] = {(cuuint64_t)sb.Kp * 2, (cuuint64_t)sb.rows * sb.Kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)OZ_BM, (cuuint32_t)sb.ns};
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

int slice_kpad(int k) { return (k + OZ_BK - 1) / OZ_BK * OZ_BK; }

size_t slice_buf_bytes(int rows, int k, int ns) { return (size_t)ns * rows * slice_kpad(k) * 2; }


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
    static const cudaError_t attr =
        cudaFuncSetAttribute(ozaki_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES);
    DME_CUDA_TRY(attr);
    const int tmt = (p.M + OZ_BM - 1) / OZ_BM, tnt = (p.N + OZ_BN - 1) / OZ_BN;
    p.tiles_n = tnt;
    const int tiles = p.tri ? tnt * (tnt + 1) / 2 : tmt * tnt;
    // split K of the last partial wave in two when it fills at most half of the SMs:
    // the wave then takes about half a tile time instead of a whole one
    static const int nsm = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return std::max(c, 1);
    }();
    const int tail = tiles % nsm;
    p.split_parts = 1;
    p.split_first = tiles;
    if (p.ws && p.ws_cnt && tiles > nsm && tail > 0 && tail <= OZ_SPLIT_MAX_TAIL && tail <= nsm / 2 &&
        p.Kp / OZ_BK >= 16) {
        p.split_parts = 2;
        p.split_first = tiles - tail;
    } else if (p.ws && p.ws_cnt && tiles <= nsm / 2 && tiles <= OZ_SPLIT_MAX_TAIL && p.Kp / OZ_BK >= 16) {
        // a single partial wave (skinny products): up to 4 K parts, at least 8 K blocks each,
        // within the SM count and the workspace's 2 x OZ_SPLIT_MAX_TAIL tile slots
        int parts = 1;
        while (parts < 4 && tiles * (parts * 2) <= nsm && tiles * (parts * 2) <= 2 * OZ_SPLIT_MAX_TAIL &&
               p.Kp / OZ_BK / (parts * 2) >= 8)
            parts *= 2;
        if (parts > 1) {
            p.split_parts = parts;
            p.split_first = 0;
        }
    }
    const int grid = p.split_first + (tiles - p.split_first) * p.split_parts;
    ozaki_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM_BYTES, st>>>(tA, tB, p);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

dme_status ozaki_grouped_prepare() {
    static const cudaError_t attr =
        cudaFuncSetAttribute(ozaki_gemm_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES);
    DME_CUDA_TRY(attr);
    return DME_OK;
}

dme_status launch_ozaki_grouped(std::vector<OzGroupDesc>& items, OzGroupDesc* dev_desc, cudaStream_t st,
                                DescArena* arena) {
    int total = 0;
    std::vector<OzGroupDesc> live;
    for (auto& it : items) {
        OzParams& p = it.p;
        if (p.M <= 0 || p.N <= 0) continue;
        if (p.Kp % OZ_BK != 0 || p.Kp > OZ_MAX_K || (p.tri && p.M != p.N)) {
            set_error("ozaki grouped gemm: bad problem shape");
            return DME_EINVAL;
        }
        const int tmt = (p.M + OZ_BM - 1) / OZ_BM, tnt = (p.N + OZ_BN - 1) / OZ_BN;
        p.tiles_n = tnt;
        it.start = total;
        total += p.tri ? tnt * (tnt + 1) / 2 : tmt * tnt;
        live.push_back(it);
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
    ozaki_gemm_grouped_kernel<<<total, OZ_THREADS, OZ_SMEM_BYTES, st>>>(d, (int)live.size());
    DME_CUDA_TRY(cudaGetLastError());
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
        const size_t off_b = off_a + align256(slice_buf_bytes(M, K, OZ_SLICES_A));
        const size_t need = off_b + align256(slice_buf_bytes(N, K, OZ_SLICES_B));
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
        sa.ns = OZ_SLICES_A;
        sa.scale = reinterpret_cast<float*>(base + off_sa);
        sa.data = reinterpret_cast<__nv_bfloat16*>(base + off_a);
        sb.rows = N;
        sb.k = K;
        sb.Kp = Kp;
        sb.ns = OZ_SLICES_B;
        sb.scale = reinterpret_cast<float*>(base + off_sb);
        sb.data = reinterpret_cast<__nv_bfloat16*>(base + off_b);
        DME_TRY(make_slice_tmap(sa, &sa.tmap));
        DME_TRY(make_slice_tmap(sb, &sb.tmap));
        // the array keeps the previous call's contents: the status word must start at zero
        // (slices, padding and scales are rewritten in full below)
        DME_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
        launch_slice_rows_f64(A, M, K, K, sa, st);
        launch_slice_rows_f64(B, N, K, K, sb, st);
        OzParams o;
        std::memset(&o, 0, sizeof(o));
        o.M = M;
        o.N = N;
        o.Kp = Kp;
        o.sa = sa.scale;
        o.sb = sb.scale;
        o.mode = OZ_OUT_F64;
        o.ldc = N;
        o.Cd = C;
        o.alpha = 1.0;
        o.status = status;
        DME_TRY(launch_ozaki_gemm(sa.tmap, sb.tmap, o, st));
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
