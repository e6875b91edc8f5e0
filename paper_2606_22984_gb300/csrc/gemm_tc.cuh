// gemm_tc.cuh -- tensor-core (tcgen05) GEMMs over "tiled" BF16 operands.
//
// Tiled layout T(rows, K): a matrix of `rows` x `K` BF16 values, rows padded
// to a multiple of 128 and K to a multiple of 64, stored as 16 KB tiles of
// 128 rows x 64 K.  Tile (rb, kc) sits at byte (kc * RB + rb) * 16384 with
// RB = ceil(rows / 128); inside a tile the core-matrix layout of tc.cuh
// (KG = 8).  One tile is one bulk copy, and the tiles of one K chunk are
// adjacent, so a B operand of up to 256 rows is one descriptor.
#pragma once

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

enum TcEpilogue {
    TE_STORE_F32 = 0,   // out_f32 = acc (+ bias)
    TE_RESID_F32 = 1,   // out_f32 = resid + acc + bias
    TE_GELU_T = 2,      // v = acc + bias: out_t = gelu(v), out_t2 = v (both tiled BF16)
    TE_GELU_BWD_T = 3,  // out_t = acc * gelu'(aux_t) (tiled BF16)
    TE_STORE_F32_T = 4, // out_f32 = acc + bias and out_t = same (tiled BF16)
};

struct RowGemm {
    const unsigned char *A;   // T(R, K)
    int64_t RB;               // row blocks of A (and of tiled outputs)
    int KC;                   // K chunks of 64
    const unsigned char *Bw;  // T(N, K): NBw row blocks
    int NBw;
    int N;                    // output columns (multiple of 32)
    int64_t R;                // valid rows
    const float *bias;        // [N] or nullptr
    float *out_f32;
    int ld_out;
    const float *resid;
    int ld_resid;
    unsigned char *out_t;     // T(R, N)
    unsigned char *out_t2;    // T(R, N)
    const unsigned char *aux_t;
    int *err;
};

struct WgradGemm {
    const unsigned char *A;   // T(M, Kr): rows = M output features, K = rows of the batch
    int64_t MB;               // row blocks of A
    const unsigned char *Bm;  // T(N, Kr)
    int NB;                   // row blocks of B
    int N;
    int M;
    int64_t KCtot;            // K chunks (ceil(Kr / 64))
    int64_t kc_per_cta;
    float *C;                 // [M][N] accumulated with atomics
    int *err;
};

sg_status launch_row_gemm(const RowGemm &g, int epi, cudaStream_t st);
sg_status launch_wgrad_gemm(const WgradGemm &g, cudaStream_t st);

// FP32 row-major [R][F] -> T(R, F) or the transpose T(F, R) (zero padding).
sg_status launch_to_tiled(const float *X, int64_t R, int F, int ldx, unsigned char *dst,
                          bool transpose, cudaStream_t st);
// T(R, F) -> T(F, R)
sg_status launch_tiled_transpose(const unsigned char *src, int64_t R, int F, unsigned char *dst,
                                 cudaStream_t st);
// FP32 row-major W[rows][K] -> T(rows, K) (weights), or of W^T when transpose.
sg_status launch_pack_tiled(const float *W, int rows, int K, unsigned char *dst, bool transpose,
                            cudaStream_t st);

}  // namespace sg
