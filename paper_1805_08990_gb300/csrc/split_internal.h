// Declarations of the split-precision (bf16 slice) path shared by libdme units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "dme_internal.h"

namespace dme {

// Digit schemes of the error-free slicing.  Both start with a leading digit
// |d0| <= 64 of weight 2^-6 (so the fp32 sum of K <= 4096 leading products is
// exact); the trailing digits are
//   OZ_DIG9: base 2^9, |d| <= 256 (every integer up to 256 is a bf16), weight
//            2^(-6-9t): four slices leave 2^-34 of the row scale, five 2^-43.
//            The per-step path: only its leading level needs exact sums.
//   OZ_DIG7: base 2^7, |d| <= 64, weight 2^(-6-7t): six slices leave 2^-42.
//            The accurate mode (Pade chain): with 7-bit digits every level
//            l <= 2 of a K chunk of 512 sums exactly in fp32.
enum { OZ_DIG9 = 9, OZ_DIG7 = 7 };

constexpr int OZ_SLICES_FIXED = 5;  // DIG9 slices of a fixed operand (E^T, S, Bt^T, A of dme_gemm_split)
constexpr int OZ_SLICES_STEP = 4;   // DIG9 slices of a per-step operand (P, U, Y, B of dme_gemm_split)
constexpr int OZ_SLICES_ACC = 6;    // DIG7 slices of the accurate mode (both operands)
constexpr int OZ_MAX_K = 4096;      // exact level-0 accumulation needs K * 64 * 64 <= 2^24
constexpr int OZ_ACC_CHUNK_KB = 16; // accurate mode: K blocks of 32 per exactly summed chunk (K = 512)

// Slice-pair configurations of the tensor kernel.  A pair (s, t) multiplies
// slice s of A by slice t of B; pairs with s + t > L are dropped.  Levels 0, 1
// and 2 have TMEM accumulators of their own, levels >= 3 share the fourth.
//   OZ_P10: A 4, B 4, L 3 (DIG9) - 10 pairs
//   OZ_P13: A 4, B 4, L 4 (DIG9) - 13 pairs
//   OZ_P14: A 5, B 4, L 4 (DIG9) - 14 pairs
//   OZ_A21: A 6, B 6, L 5 (DIG7) - 21 pairs, K in exact chunks of 512,
//           chunk sums combined in fp64 (accurate mode)
enum OzCfgId { OZ_P10 = 0, OZ_P13 = 1, OZ_P14 = 2, OZ_A21 = 3, OZ_NCFG = 4 };
int oz_cfg_pairs(int cfg);          // slice products per output
int oz_cfg_slices_a(int cfg);
int oz_cfg_slices_b(int cfg);
int oz_cfg_scheme(int cfg);         // OZ_DIG9 or OZ_DIG7
enum { OZ_OUT_PAIR = 0, OZ_OUT_F64 = 1 };

// Slices of a rows x k operand: planes [ns][rows][Kp] bf16 (Kp = k rounded
// up to 32, zero padded) and one power-of-two scale per row.  A tensor-map load
// brings a 32 x 128 tile of every plane a configuration reads (box 32 x 128 x
// planes): tmap spans all ns planes, tmap4 the first four (when ns > 4).
struct SliceBuf {
    __nv_bfloat16* data = nullptr;
    float* scale = nullptr;
    int rows = 0, k = 0, Kp = 0, ns = 0;
    int scheme = OZ_DIG9;
    CUtensorMap tmap;
    CUtensorMap tmap4;
};

struct OzParams {
    int M, N, Kp;
    int cfg;              // OzCfgId
    const float* sa;      // row scales of A (M)
    const float* sb;      // row scales of B (N)
    int mode;             // OZ_OUT_PAIR or OZ_OUT_F64
    int tri;              // OZ_OUT_F64 only: upper tiles, mirrored (M == N); addends symmetric
    int ldc;
    float2* Cp;           // OZ_OUT_PAIR output (normalised hi, lo)
    double* Cd;           // OZ_OUT_F64 output
    double alpha;         // OZ_OUT_F64: v = alpha acc + b1 D1 + b2 D2 + b3 D3
    const double* D1;
    const double* D2;
    const double* D3;
    double b1, b2, b3;
    int tiles_n;          // set by the launcher
    int tiles;            // set by the launcher
    int units;            // set by the launcher
    int* status;
    // split-K of the last partial wave (single-problem launches only): tiles with index
    // >= split_first run as split_parts units over consecutive K ranges; each writes its
    // level sums to ws, and a second kernel adds them in part order and runs the
    // epilogue.  ws: [tail tile][part][128 x 128] (level 0, levels >= 1).
    float2* ws;
    int* ws_cnt;          // unused (kept for the layout of the grouped descriptors)
    int split_first;      // set by the launcher
    int split_parts;      // set by the launcher (1: no split)
    // accurate mode: [chunk][M][N] doubles of the per-chunk products (chunks of
    // OZ_ACC_CHUNK_KB K blocks), summed in chunk order by a second kernel into Cd
    double* wsd;
    int nchunks;          // set by the launcher
};

constexpr int OZ_SPLIT_MAX_TAIL = 76;     // tail tiles that may be split (half of 152 SMs)
constexpr size_t OZ_SPLIT_WS_FLOAT2 = (size_t)OZ_SPLIT_MAX_TAIL * 2 * 128 * 128;

// One problem of a grouped split GEMM (tensor maps live in global memory).
struct OzGroupDesc {
    CUtensorMap tmA;
    CUtensorMap tmB;
    OzParams p;
    int start;            // first unit index (set by the launcher)
    int tail_start;       // first split tile in the launch's tail kernel (set by the launcher)
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
// Encode sb.tmap and (ns > 4) sb.tmap4.
dme_status make_slice_tmaps(SliceBuf& sb);
// The tensor map of A's (or B's) slices whose box spans the planes configuration cfg reads.
inline const CUtensorMap& oz_tmap_a(const SliceBuf& A, int cfg) {
    return A.ns > oz_cfg_slices_a(cfg) ? A.tmap4 : A.tmap;
}
inline const CUtensorMap& oz_tmap_b(const SliceBuf& B, int cfg) {
    return B.ns > oz_cfg_slices_b(cfg) ? B.tmap4 : B.tmap;
}
// Slice the rows of X (rows x cols, leading dimension ldx; rows <= sb.rows) into sb
// (planes and digit scheme of sb: DIG9 with 4 or 5, DIG7 with 6; each plane holds
// sb.rows rows, the ones past `rows` untouched).
void launch_slice_rows_f64(const double* X, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st);
void launch_slice_rows_pair(const float2* Xp, int rows, int cols, int ldx, const SliceBuf& sb, cudaStream_t st);
// One launch slicing the rows of every item (4 DIG9 slices each; pair: the items are
// (hi, lo) float pairs, else FP64), descriptors staged in the arena.
dme_status launch_slice_grouped(std::vector<SliceDesc>& items, bool pair, cudaStream_t st, DescArena* arena);
// OzParams for C = A B^T from two slice buffers under configuration cfg (checks that
// the buffers hold the slices and scheme the configuration reads).
dme_status oz_params(const SliceBuf& A, const SliceBuf& B, int cfg, OzParams* p);
// The accurate mode's chunk workspace in doubles for an M x N product over K.
size_t oz_acc_ws_doubles(int M, int N, int K);
dme_status launch_ozaki_gemm(const CUtensorMap& tA, const CUtensorMap& tB, OzParams p, cudaStream_t st);
// Grouped launch over independent problems: items of 10 and 13 slice products
// together, or of 14 alone (not the accurate mode), ordered by K per unit,
// largest first, so that the longest units start in the first wave.  A problem
// with a workspace (p.ws) splits K by the same rule as its single-problem
// launch (and gives the same bits); one tail launch adds the parts of every
// split problem.  dev_desc holds items.size() descriptors.
// Set the grouped kernel's shared-memory attribute (before any stream capture).
dme_status ozaki_grouped_prepare();
// With `arena` the descriptors are staged there instead of copied to dev_desc.
dme_status launch_ozaki_grouped(std::vector<OzGroupDesc>& items, OzGroupDesc* dev_desc, cudaStream_t st,
                                DescArena* arena = nullptr);

}  // namespace dme
