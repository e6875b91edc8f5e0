// gemm_tc.cuh -- tensor-core (tcgen05) GEMMs over "tiled" BF16 operands.
//
// Tiled layout T(rows, K): a matrix of `rows` x `K` BF16 values, rows padded
// to a multiple of 128 and K to a multiple of 64, stored as 16 KB tiles of
// 128 rows x 64 K.  Tile (rb, kc) sits at byte (kc * RB + rb) * 16384 with
// RB = ceil(rows / 128); inside a tile the core-matrix layout of tc.cuh
// (KG = 8).  One tile is one bulk copy, and the tiles of one K chunk are
// adjacent, so a B operand of up to 256 rows is one descriptor.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "sg_internal.cuh"
#include "tc.cuh"

namespace sg {

constexpr int kTileBytes = 128 * 64 * 2;

__host__ __device__ __forceinline__ int64_t tl_blocks(int64_t rows) { return (rows + 127) >> 7; }

__host__ __device__ __forceinline__ size_t tl_bytes(int64_t rows, int K)
{
    return (size_t)tl_blocks(rows) * ((K + 63) >> 6) * kTileBytes;
}

// Byte offset of element (r, k) in T(rows, K) with RB row blocks.
__host__ __device__ __forceinline__ size_t tl_offset(int64_t r, int k, int64_t RB)
{
    return ((size_t)((int64_t)(k >> 6) * RB + (r >> 7)) << 14) +
           tc::cm_offset((int)(r & 127), k & 63, 8);
}

// Wide layout W(R, F) of activations: row block rb (128 rows) is one [128 x F]
// core-matrix tile (KG = F / 8) at byte rb * 256 F, so a row block is one
// bulk copy.  Read K-major (K = F) by the row GEMMs: descriptor strides 128 B
// along K and 16 F bytes between 8-row groups.  Read MN-major (MN = F, K =
// rows) by the weight-gradient GEMM: 128 B along MN and 16 F bytes along K.
// Rows past R up to the block end are zero; a slack tail lets a 128-wide
// operand window that overhangs F stay inside the buffer.  F is a multiple of 16.
constexpr size_t kWideSlack = 4096;

__host__ __device__ __forceinline__ size_t wl_block_bytes(int F) { return (size_t)256 * F; }

__host__ __device__ __forceinline__ size_t wl_bytes(int64_t R, int F)
{
    return (size_t)tl_blocks(R) * wl_block_bytes(F) + kWideSlack;
}

__host__ __device__ __forceinline__ size_t wl_offset(int64_t r, int f, int F)
{
    return (size_t)(r >> 7) * wl_block_bytes(F) + tc::cm_offset((int)(r & 127), f, F >> 3);
}

enum TcEpilogue {
    TE_STORE_F32 = 0,   // out_f32 = acc (+ bias)
    TE_RESID_F32 = 1,   // out_f32 = resid + acc + bias
    TE_GELU_T = 2,      // v = acc + bias: out_t = gelu(v), out_t2 = gelu'(v) (both wide BF16; out_t2 optional)
    TE_GELU_BWD_T = 3,  // out_t = acc * aux_t, aux_t = gelu'(v) from the forward (wide BF16)
    TE_STORE_F32_T = 4, // out_f32 = acc + bias and out_t = same (tiled BF16)
    TE_STORE_BF16 = 5,  // out_h = acc + bias, row-major BF16 (ld_out elements per row)
    TE_LN_BWD = 6,      // acc = dY of a LayerNorm: out_f32 = dX (+ ln_dres), its wide copy
                        // ln_dxt, dg/db/dcol column sums (N in {32, 64, 128, 256})
};

struct RowGemm {
    const unsigned char *A;   // W(R, K)
    int64_t RB;               // row blocks of A (and of the wide outputs)
    int K;                    // reduction length (multiple of 16)
    int KC;                   // K chunks of 64 of the weights
    const unsigned char *Bw;  // T(N, K): NBw row blocks
    int NBw;
    int N;                    // output columns (multiple of 32)
    int64_t R;                // valid rows
    const float *bias;        // [N] or nullptr
    float *out_f32;
    int ld_out;
    const float *resid;
    int ld_resid;
    unsigned char *out_t;     // W(R, N)
    __nv_bfloat16 *out_h;     // row-major BF16 [R][ld_out]
    unsigned char *out_t2;    // W(R, N)
    const unsigned char *aux_t;  // W(R, N)
    float *colsum;            // TE_GELU_BWD_T: colsum[j] += sum_r out(r, j) (N <= 1024), or nullptr
    int staged;               // set by the launcher: row-major outputs through shared memory
    // TE_LN_BWD: the LayerNorm y = (x - mu) rs g + b whose input gradient this
    // product's output dY feeds: dX = ln_dres + rs (dY g - mean(dY g) - xhat
    // mean(dY g xhat)); ln_dg += sum dY xhat, ln_db += sum dY, ln_dcol += sum dX
    const float *ln_x, *ln_mu, *ln_rs, *ln_g, *ln_dres;
    float *ln_dg, *ln_db, *ln_dcol;
    unsigned char *ln_dxt;    // W(R, N) copy of dX (rows past R zero), or nullptr
    int *err;
};

// C += A^T B over the rows of two wide activations (both operands MN-major):
// C[m][n] = sum_r A[r][m] B[r][n], or stored at C[n][m] when transpose_out.
struct WgradGemm {
    const unsigned char *A;   // W(R, M)
    int M;
    const unsigned char *Bm;  // W(R, N)
    int N;
    int64_t RB;               // row blocks (the reduction, 128 rows each)
    int64_t rb_per_cta;       // row blocks per split
    float *C;
    int ldc;
    int transpose_out;
    int *err;
};

sg_status launch_row_gemm(const RowGemm &g, int epi, cudaStream_t st);
// Whether launch_row_gemm(g, TE_LN_BWD) can run for g's shape.
bool ln_bwd_fusable(const RowGemm &g);
sg_status launch_wgrad_gemm(const WgradGemm &g, cudaStream_t st);

// FP32 row-major [R][F] -> T(R, F) or the transpose T(F, R) (zero padding).
sg_status launch_to_tiled(const float *X, int64_t R, int F, int ldx, unsigned char *dst,
                          bool transpose, cudaStream_t st);
// FP32 row-major [R][F] -> W(R, F) (rows past R zero).
sg_status launch_to_wide(const float *X, int64_t R, int F, unsigned char *dst, cudaStream_t st);
// Rows past R up to the end of the last row block of W(R, F) set to zero.
sg_status launch_zero_wide_tail(int64_t R, int F, unsigned char *dst, cudaStream_t st);
// FP32 row-major W[rows][K] -> T(rows, K) (weights), or of W^T when transpose.
sg_status launch_pack_tiled(const float *W, int rows, int K, unsigned char *dst, bool transpose,
                            cudaStream_t st);

}  // namespace sg
