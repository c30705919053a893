// lu_internal.cuh -- launch constants and the work-buffer map shared by the
// library's host drivers.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace mw {

constexpr int kPanelThreads = 256;
constexpr int kPanelRowsPerCta = 8;    // panel rows per CTA before adding CTAs
constexpr int kMaxPanelCtas = 256;
constexpr int kDefaultNb = 64;          // panel width of the blocked LU
constexpr int kMaxNb = 128;

// LU work buffer: [barrier | status | panel candidates | split-update scratch]
// The candidate area holds, for two column parities, one record per CTA
// (the candidate value, its row index and a copy of the whole candidate row
// of the panel) and a copy of the old row k.
constexpr size_t kWsBarrier = 0;
constexpr size_t kWsStatus = 64;
constexpr size_t kWsCand = 256;
constexpr size_t kCandStride = 8 * (4 + 1 + 4 * kMaxNb);             // doubles of one record, in bytes
constexpr size_t kCandParity = kCandStride * kMaxPanelCtas + 8 * 4 * kMaxNb;  // records + old row k
constexpr size_t kWsSplit = (kWsCand + 2 * kCandParity + 65535) & ~(size_t)65535;

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// tuning knobs (capi.cu): value of `param` (MW_TUNE_*) for precision prec
int tune_get(int param, int prec);

template <int W>
int lu_blocked(int update, int64_t n, double* A, int64_t lda, int64_t* piv, int64_t* info,
               char* ws, size_t ws_bytes, int nb, cudaStream_t s);

// split-precision trailing update for DD (ozaki.cu): C -= L21 * U12
int split_update_dd(double* A, int64_t lda, int64_t plane, int64_t row0, int64_t m,
                    int64_t col0, int64_t N, int64_t k0, int nb, char* ws, size_t ws_bytes,
                    cudaStream_t s);
size_t split_workspace_bytes(int64_t n, int nb);
int split_gemm_sub_dd(int64_t m, int64_t N, double* C, int64_t ldc, int64_t planeC, const double* L,
                      int64_t ldl, int64_t planeL, const double* U, int64_t ldu, int64_t planeU,
                      char* ws, size_t ws_bytes, cudaStream_t s);
template <int W>
int launch_gemm_plain_ptr(int64_t m, int64_t N, int K, double* C, int64_t ldc, int64_t planeC,
                          const double* L, int64_t ldl, int64_t planeL, const double* U, int64_t ldu,
                          int64_t planeU, cudaStream_t s);

// substitution (solve.cu); y is a w-plane vector work area of n
template <int W>
int solve_launch(int64_t n, const double* LU, int64_t lda, const int64_t* piv, const double* b,
                 double* x, char* ws, size_t ws_bytes, cudaStream_t s);
size_t solve_workspace_bytes(int w, int64_t n);

// exact residual (residual.cu)
int residual_launch(int64_t n, const double* A, int64_t lda, int a_words, const double* b,
                    int b_words, const double* x, int x_words, double* r, int r_words,
                    cudaStream_t s);

}  // namespace mw
