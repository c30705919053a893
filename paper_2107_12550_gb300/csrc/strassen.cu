// strassen.cu -- C = A B for square multiword matrices by Strassen's
// recursion over the block matrix product: the paper's second matmul
// (Section 2, the Strassen form of BNCmatmul).
//
// Per level, with the quadrants X11, X12, X21, X22 of each operand and every
// + / - one rounded multiword addition or subtraction, in this order:
//   M1 = (A11 + A22)(B11 + B22)     M5 = (A11 + A12) B22
//   M2 = (A21 + A22) B11            M6 = (A21 - A11)(B11 + B12)
//   M3 = A11 (B12 - B22)            M7 = (A12 - A22)(B21 + B22)
//   M4 = A22 (B21 - B11)
//   C11 = ((M1 + M4) - M5) + M7     C12 = M3 + M5
//   C21 = M2 + M4                   C22 = ((M1 - M2) + M3) + M6
// (Strassen 1969).  At the last level each product is the block matrix
// product from a zero C: the plain form (c = c + a_t b_t in ascending t) or
// the split form (per 64-wide slab, the exact slab product added and rounded
// to DD).  Seven products per level instead of eight: 7/8 of the
// multiply-adds per level, at the price of 18 matrix additions and a larger
// error bound than the classical product.
#include <cuda_runtime.h>
#include <cstdint>

#include "mw_arith.cuh"
#include "mw_common.cuh"
#include "lu_internal.cuh"

namespace mw {

// Z = X + Y or X - Y on an m x n block (column-major, w planes); Z may be X
template <int W>
__global__ void __launch_bounds__(256)
k_madd(int subtract, int64_t m, const double* X, int64_t ldx, int64_t px, const double* Y, int64_t ldy,
       int64_t py, double* Z, int64_t ldz, int64_t pz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (i >= m) return;
  const val<W> x = load<W>(X, px, j * ldx + i);
  const val<W> y = load<W>(Y, py, j * ldy + i);
  store<W>(Z, pz, j * ldz + i, subtract ? sub<W>(x, y) : add<W>(x, y));
}

namespace {

struct Mat {
  double* p;
  int64_t ld, plane;
};

template <int W>
int madd(int subtract, int64_t h, const Mat& X, const Mat& Y, const Mat& Z, cudaStream_t s) {
  k_madd<W><<<dim3((unsigned)((h + 255) / 256), (unsigned)h), 256, 0, s>>>(subtract, h, X.p, X.ld, X.plane, Y.p,
                                                                         Y.ld, Y.plane, Z.p, Z.ld, Z.plane);
  MW_LAUNCH_CHECK();
  return MW_OK;
}

// C = A B (h x h) by the block matrix product from a zero C
template <int W>
int base_product(int update, int64_t h, const Mat& A, const Mat& B, const Mat& C, char* split_ws,
                 size_t split_bytes, cudaStream_t s) {
  for (int c = 0; c < W; ++c)
    MW_CUDA_CHECK(cudaMemset2DAsync(C.p + c * C.plane, sizeof(double) * C.ld, 0, sizeof(double) * h, h, s));
  if (update == MW_UPDATE_PLAIN)
    return launch_gemm_plain_ptr<W>(h, h, (int)h, C.p, C.ld, C.plane, A.p, A.ld, A.plane, B.p, B.ld, B.plane, s,
                                    true);
  for (int64_t k0 = 0; k0 < h; k0 += kDefaultNb) {
    const int rc = split_gemm_sub_dd(h, h, C.p, C.ld, C.plane, A.p + k0 * A.ld, A.ld, A.plane, B.p + k0, B.ld,
                                     B.plane, split_ws, split_bytes, s, true);
    if (rc) return rc;
  }
  return MW_OK;
}

// the recursion; tmp holds 9 h^2 w doubles for this level, then the deeper
// levels' temporaries
template <int W>
int strassen_rec(int update, int levels, int64_t n, const Mat& A, const Mat& B, const Mat& C, double* tmp,
                 char* split_ws, size_t split_bytes, cudaStream_t s) {
  if (levels == 0) return base_product<W>(update, n, A, B, C, split_ws, split_bytes, s);
  const int64_t h = n / 2, hh = h * h;
  auto quad = [&](const Mat& X, int r, int c) { return Mat{X.p + c * h * X.ld + r * h, X.ld, X.plane}; };
  auto tmat = [&](int k) { return Mat{tmp + (size_t)k * W * hh, h, hh}; };
  const Mat A11 = quad(A, 0, 0), A12 = quad(A, 0, 1), A21 = quad(A, 1, 0), A22 = quad(A, 1, 1);
  const Mat B11 = quad(B, 0, 0), B12 = quad(B, 0, 1), B21 = quad(B, 1, 0), B22 = quad(B, 1, 1);
  const Mat C11 = quad(C, 0, 0), C12 = quad(C, 0, 1), C21 = quad(C, 1, 0), C22 = quad(C, 1, 1);
  const Mat S = tmat(0), T = tmat(1);
  Mat M[7];
  for (int k = 0; k < 7; ++k) M[k] = tmat(2 + k);
  double* deeper = tmp + (size_t)9 * W * hh;
  auto rec = [&](const Mat& X, const Mat& Y, const Mat& Z) {
    return strassen_rec<W>(update, levels - 1, h, X, Y, Z, deeper, split_ws, split_bytes, s);
  };
  int rc;
#define MW_TRY(expr)   \
  if ((rc = (expr))) { \
    return rc;         \
  }
  MW_TRY(madd<W>(0, h, A11, A22, S, s));
  MW_TRY(madd<W>(0, h, B11, B22, T, s));
  MW_TRY(rec(S, T, M[0]));
  MW_TRY(madd<W>(0, h, A21, A22, S, s));
  MW_TRY(rec(S, B11, M[1]));
  MW_TRY(madd<W>(1, h, B12, B22, T, s));
  MW_TRY(rec(A11, T, M[2]));
  MW_TRY(madd<W>(1, h, B21, B11, T, s));
  MW_TRY(rec(A22, T, M[3]));
  MW_TRY(madd<W>(0, h, A11, A12, S, s));
  MW_TRY(rec(S, B22, M[4]));
  MW_TRY(madd<W>(1, h, A21, A11, S, s));
  MW_TRY(madd<W>(0, h, B11, B12, T, s));
  MW_TRY(rec(S, T, M[5]));
  MW_TRY(madd<W>(1, h, A12, A22, S, s));
  MW_TRY(madd<W>(0, h, B21, B22, T, s));
  MW_TRY(rec(S, T, M[6]));
  MW_TRY(madd<W>(0, h, M[0], M[3], C11, s));
  MW_TRY(madd<W>(1, h, C11, M[4], C11, s));
  MW_TRY(madd<W>(0, h, C11, M[6], C11, s));
  MW_TRY(madd<W>(0, h, M[2], M[4], C12, s));
  MW_TRY(madd<W>(0, h, M[1], M[3], C21, s));
  MW_TRY(madd<W>(1, h, M[0], M[1], C22, s));
  MW_TRY(madd<W>(0, h, C22, M[2], C22, s));
  MW_TRY(madd<W>(0, h, C22, M[5], C22, s));
#undef MW_TRY
  return MW_OK;
}

}  // namespace

size_t strassen_split_bytes(int update, int levels, int64_t n) {
  return update == MW_UPDATE_SPLIT ? align256(256 + split_workspace_bytes(n >> levels, kDefaultNb)) : 256;
}

size_t strassen_workspace_bytes(int w, int update, int levels, int64_t n) {
  size_t doubles = 0;
  for (int l = 1; l <= levels; ++l) {
    const size_t h = (size_t)(n >> l);
    doubles += (size_t)9 * (size_t)w * h * h;
  }
  return strassen_split_bytes(update, levels, n) + sizeof(double) * doubles;
}

int strassen_run(int w, int update, int levels, int64_t n, const double* A, int64_t lda, const double* B,
                 int64_t ldb, double* C, int64_t ldc, char* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < strassen_workspace_bytes(w, update, levels, n)) return MW_EUNSUPPORTED;
  const size_t sb = strassen_split_bytes(update, levels, n);
  double* tmp = reinterpret_cast<double*>(ws + sb);
  const Mat Am{const_cast<double*>(A), lda, lda * n}, Bm{const_cast<double*>(B), ldb, ldb * n}, Cm{C, ldc, ldc * n};
  switch (w) {
    case 2: return strassen_rec<2>(update, levels, n, Am, Bm, Cm, tmp, ws, sb, s);
    case 3: return strassen_rec<3>(update, levels, n, Am, Bm, Cm, tmp, ws, sb, s);
    default: return strassen_rec<4>(update, levels, n, Am, Bm, Cm, tmp, ws, sb, s);
  }
}

}  // namespace mw
