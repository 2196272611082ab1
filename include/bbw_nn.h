/*
 * bbw_nn.h -- C ABI of the neural-operator surrogate's GPU kernels
 * (libbbwadg.so). The paper has no counterpart: the surrogate is a learned
 * map from a c^2 field and a source position to receiver traces, trained on
 * runs of this library's BBWADG solver, which also measures its error and is its
 * fallback. The network is composed from these calls (binding: surrogate.py).
 *
 * All pointers are caller-owned device memory (FP32 unless stated); every call
 * is asynchronous on `stream` (cudaStream_t, NULL = legacy default stream) and
 * returns a bbw_status (declared in bbwadg.h); errors set bbw_last_error().
 */
#ifndef BBW_NN_H
#define BBW_NN_H

#include "bbwadg.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Batched GEMM on the BF16 tensor cores with FP32 accumulation:
 *   C[b] = alpha op(A[b]) op(B[b]) + beta C[b] (+ bias[n]),  b < batch,
 * op(A) M x K, op(B) K x N, all row-major. transA = 0: A is M x K with leading
 * dimension lda; transA = 1: A is stored K x M. transB likewise (0: K x N,
 * 1: N x K). Batch b starts at A + b strideA, B + b strideB, C + b strideC
 * (elements; a stride of 0 shares the matrix). A and B are rounded to BF16.
 * Epilogue: bias (length N, may be NULL); pre (may be NULL, laid out like C)
 * receives the value before the activation; act = 0 (none) or 1 (GELU, the
 * erf form). splits > 1 divides K among that many thread blocks that add their
 * partial products atomically into C (for very long K, e.g. weight gradients);
 * then bias, pre, act must be unset and beta 0 (C accumulates: clear it
 * first; the order of the atomic additions, and so the last bits of C, may
 * differ between calls). splits <= 1024. An operand whose rows start on 16
 * bytes (leading dimension and stride multiples of 4 floats, 16-byte base)
 * is loaded 16 bytes at a time, otherwise element by element (same result).
 * Errors: BBW_ERR_ARG for bad sizes, NULL matrices or grid limits
 * (batch x splits <= 65535, M <= 64 x 65535).
 */
bbw_status bbw_nn_gemm(int M, int N, int K, const float* A, int lda, long long strideA, int transA, const float* B,
                       int ldb, long long strideB, int transB, float* C, int ldc, long long strideC, int batch,
                       float alpha, float beta, const float* bias, float* pre, int act, int splits, void* stream);

/*
 * Transform along the innermost spatial axis of `pencils` pencils with C
 * contiguous channels, by basis [L][m] (m <= 16, L m floats <= 48 KB), in
 * FP32. expand = 0 contracts: in [pencils][L][C] -> out [pencils][m][C],
 * out[k] = sum_z basis[z][k] in[z] (beta, pre, act must be 0 / NULL).
 * expand = 1 expands: in [pencils][m][C] -> out [pencils][L][C],
 * v = sum_k basis[z][k] in[k] + beta out[z], pre[z] = v (pre may be NULL),
 * out[z] = act ? GELU(v) : v (act 0 or 1). in and out must not overlap.
 */
bbw_status bbw_nn_axis_transform(const float* basis, int L, int m, const float* in, float* out, long long pencils,
                                 int C, int expand, float beta, float* pre, int act, void* stream);

/* grad[i] *= GELU'(pre[i]) for i < n (the backward of the GELU epilogue). */
bbw_status bbw_nn_gelu_backward(const float* pre, float* grad, long long n, void* stream);

/* db[j] += sum_i dY[i][j] over rows i < rows of dY [rows][N]. */
bbw_status bbw_nn_bias_grad(const float* dY, float* db, long long rows, int N, void* stream);

/*
 * Receiver features from a field u [B][X][Y][Z][C]: out [B][R][C] is the mean
 * of the eight grid points (rx[r] + {0,1}, ry[r] + {0,1}, rz[r] + {0,1})
 * (int device arrays rx, ry, rz [R]; the stencils of different receivers must
 * be disjoint; a stencil not inside the grid gives 0). transpose = 1 applies
 * the transpose instead: u += the scatter of out (the backward).
 */
bbw_status bbw_nn_gather_receivers(const float* u, float* out, const int* rx, const int* ry, const int* rz, int B,
                                   int X, int Y, int Z, int C, int R, int transpose, void* stream);

/*
 * Time-shifted traces: out[i][t] = scale[i] * in[i](t + shift[i]) for rows
 * i < rows of T samples, in[i](x) the linear interpolation, at the fractional
 * position x, of the samples extended by zeros (in[i][j] = 0 for j < 0 or
 * j >= T). shift [rows] (samples, any sign), scale [rows] (NULL: 1); in and
 * out must not be the same array.
 */
bbw_status bbw_nn_shift_traces(const float* in, float* out, const float* shift, const float* scale, long long rows,
                               int T, void* stream);

/* loss[0] += sum_i (y_i - t_i)^2 / n and, if dy != NULL, dy = 2 (y - t) / n. */
bbw_status bbw_nn_mse(const float* y, const float* t, float* dy, float* loss, long long n, void* stream);

/* One Adam step (Kingma & Ba) of parameters p with gradient g and moments m,
 * v (all length n), step >= 1, learning rate lr, decay rates b1, b2, eps. */
bbw_status bbw_nn_adam(float* p, const float* g, float* m, float* v, long long n, int step, float lr, float b1,
                       float b2, float eps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BBW_NN_H */
