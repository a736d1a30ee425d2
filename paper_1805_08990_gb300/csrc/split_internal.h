// Declarations of the split-precision (bf16 slice) path shared by libdme units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "dme_internal.h"

namespace dme {

constexpr int OZ_SLICES_A = 5;      // bf16 slices per row of the fixed operand (E^T, S, A of dme_gemm_split)
constexpr int OZ_SLICES_B = 4;      // bf16 slices per row of the per-step operand (P, U, B)
constexpr int OZ_MAX_K = 4096;      // exact level-0 accumulation needs K * 64 * 64 <= 2^24
enum { OZ_OUT_PAIR = 0, OZ_OUT_F64 = 1 };

// Slices of a rows x k operand: planes [ns][rows][Kp] bf16 (Kp = k rounded
// up to 32, zero padded) and one power-of-two scale per row.
struct SliceBuf {
    __nv_bfloat16* data = nullptr;
    float* scale = nullptr;
    int rows = 0, k = 0, Kp = 0, ns = 0;
    CUtensorMap tmap;
};

struct OzParams {
    int M, N, Kp;
    const float* sa;      // row scales of A (M)
    const float* sb;      // row scales of B (N)
    int mode;             // OZ_OUT_PAIR or OZ_OUT_F64
    int tri;              // OZ_OUT_F64 only: upper tiles, mirrored (M == N)
    int ldc;
    float2* Cp;           // OZ_OUT_PAIR output (normalised hi, lo)
    double* Cd;           // OZ_OUT_F64 output
    double alpha;         // OZ_OUT_F64: v = alpha acc + b1 D1 + b2 D2 + b3 D3
    const double* D1;
    const double* D2;
    const double* D3;
    double b1, b2, b3;
    int tiles_n;          // set by the launcher
    int* status;
    // split-K of the last partial wave (single-problem launches only): tiles with index
    // >= split_first run as split_parts CTAs over consecutive K ranges; each writes its
    // level sums to ws and the last to arrive (counter in ws_cnt) adds them in part order
    // and runs the epilogue.  ws: [tail tile][part][128 x 128] (level 0, levels 1-4).
    float2* ws;
    int* ws_cnt;
    int split_first;      // set by the launcher
    int split_parts;      // set by the launcher (1: no split)
};

constexpr int OZ_SPLIT_MAX_TAIL = 76;     // tail tiles that may be split (half of 152 SMs)
constexpr size_t OZ_SPLIT_WS_FLOAT2 = (size_t)OZ_SPLIT_MAX_TAIL * 2 * 128 * 128;

// One problem of a grouped split GEMM (tensor maps live in global memory).
struct OzGroupDesc {
    CUtensorMap tmA;
    CUtensorMap tmB;
    OzParams p;
    int start;            // first tile index (set by the launcher)
};

// One problem of a grouped slicing launch (rows of X or of pair matrix Xp).
struct SliceDesc {
    const double* X;
    const float2* Xp;
    int rows, cols, ldx;
    __nv_bfloat16* out;
    int Kp, ns, prow;
    float* scale;
    int row0;             // set by the launcher
};

int slice_kpad(int k);
size_t slice_buf_bytes(int rows, int k, int ns);
dme_status make_slice_tmap(const SliceBuf& sb, CUtensorMap* out);
// Slice the rows of X (rows x cols, leading dimension ldx; rows <= sb.rows) into sb
// (sb.ns = 4 or 5; each plane holds sb.rows rows, the ones past `rows` untouched).
void launch_slice_rows_f64(const double* X, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st);
void launch_slice_rows_pair(const float2* Xp, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st);
// One launch slicing the rows of every item (4 slices each; pair: the items are
// (hi, lo) float pairs, else FP64), descriptors staged in the arena.
dme_status launch_slice_grouped(std::vector<SliceDesc>& items, bool pair, cudaStream_t st, DescArena* arena);
dme_status launch_ozaki_gemm(const CUtensorMap& tA, const CUtensorMap& tB, OzParams p, cudaStream_t st);
// Grouped launch over independent problems; dev_desc holds items.size() descriptors.
// Set the grouped kernel's shared-memory attribute (before any stream capture).
dme_status ozaki_grouped_prepare();
// With `arena` the descriptors are staged there instead of copied to dev_desc.
dme_status launch_ozaki_grouped(std::vector<OzGroupDesc>& items, OzGroupDesc* dev_desc, cudaStream_t st,
                                DescArena* arena = nullptr);

}  // namespace dme
