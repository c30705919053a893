// lu_internal.cuh -- launch constants and the work-buffer map shared by the
// library's host drivers.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace mw {

struct DeviceStatus;   // mw_common.cuh

constexpr int kPanelThreads = 256;
constexpr int kPanelRowsPerCta = 8;    // panel rows per CTA before adding CTAs
constexpr int kMaxPanelCtas = 256;
constexpr int kDefaultNb = 64;          // panel width of the blocked LU
constexpr int kMaxNb = 128;
constexpr size_t kPanelResidentMax = 200 * 1024;   // shared memory for panel rows kept resident

// LU work buffer: [abort word | status | panel candidates | split-update scratch]
// The candidate area holds, for two column parities, one record per CTA
// (a ready tag, the candidate value, its row index and a copy of the whole
// candidate row of the panel) and a copy of the old row k.  It is cleared at
// the start of every factorisation.
constexpr size_t kWsAbort = 0;
constexpr size_t kWsStatus = 64;
constexpr size_t kWsCand = 256;
constexpr size_t kCandStride = 8 * (1 + 4 + 1 + 4 * kMaxNb);         // one record, in bytes
constexpr size_t kCandParity = kCandStride * kMaxPanelCtas + 8 * 4 * kMaxNb;  // records + old row k
constexpr size_t kWsSplit = (kWsCand + 2 * kCandParity + 65535) & ~(size_t)65535;

// The row interchanges of one panel as a single gather: the swaps
// (k, piv[k]) for k in [k0, k0 + nb) compose to a permutation of at most 2 nb
// rows, listed as (destination, source) pairs; every column then loads all
// sources before storing all destinations.
struct SwapPlan {
  int count;
  int pad;
  int2 pairs[2 * kMaxNb];
};
constexpr size_t kWsSwapPlan = (kWsCand + 2 * kCandParity + 255) & ~(size_t)255;
static_assert(kWsSwapPlan + sizeof(SwapPlan) <= kWsSplit, "swap plan inside the LU work buffer header");

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Largest order (and leading dimension, and GEMM dimension) any
// single-system entry point accepts.  Every size computed from values up to
// this bound fits without overflow: plane strides ld * n <= 2^56 in int64,
// the refinement's LU copy 8 * 4 * n^2 <= 2^61 bytes and Strassen's
// temporaries (9 w (n/2)^2 doubles per level, summed) below 2^63 bytes in
// size_t.  An n x n multiword matrix at this order would already hold 2^56
// entries per word, far beyond any device.
constexpr int64_t kMaxOrder = (int64_t)1 << 28;

// tuning knobs (capi.cu): value of `param` (MW_TUNE_*) for precision prec
int tune_get(int param, int prec);

// The look-ahead's second stream (lu.cu): one per device, of the device's
// highest priority, with a fork and a join event; created by the first call
// that asks for it outside a stream capture.  A call holds the device's
// lock from open() until it is destroyed, so the forks and joins of calls
// from different host threads never interleave; the destructor joins a
// fork left open by an early error return, so none of the call's work runs
// after the caller's stream has passed the call.
class SideStream {
 public:
  SideStream() = default;
  SideStream(const SideStream&) = delete;
  SideStream& operator=(const SideStream&) = delete;
  ~SideStream();
  // for a call on stream s: *ready is false (with MW_OK) when the side
  // stream does not exist yet and s is capturing (the call then runs its
  // serial schedule)
  int open(cudaStream_t s, bool* ready);
  // the side stream, ordered after everything enqueued on s so far
  int fork(cudaStream_t* s2);
  // s waits for everything enqueued on the side stream so far
  int join();

 private:
  int dev_ = -1;
  cudaStream_t s_ = nullptr, s2_ = nullptr;
  cudaEvent_t fork_ = nullptr, join_ = nullptr;
  bool open_ = false;
};

template <int W>
int lu_blocked(int update, int64_t n, double* A, int64_t lda, int64_t* piv, int64_t* info,
               char* ws, size_t ws_bytes, int nb, cudaStream_t s);

// One split-precision product C -= L U (DD, ozaki.cu): entry (r, k) of L at
// L[r*lrs + k*lks], (k, j) of U at U[k*uks + j*ujs], (r, j) of C at
// C[r*crs + j*cjs]; the second word of each operand one plane further;
// inner dimension K <= 64 (the digits of k >= K are zero).
struct SplitOperands {
  const double* L;
  int64_t lrs, lks, planeL;
  const double* U;
  int64_t uks, ujs, planeU;
  double* C;
  int64_t crs, cjs, planeC;
  int64_t m, N;
  int K;
  int plus = 0;   // 1: C += L U instead of C -= L U
};
// the product on the work buffer's slice area; its tensor-core launch is
// counted under profile phase `phase`
int split_product_dd(const SplitOperands& o, char* ws, size_t ws_bytes, int phase, cudaStream_t s);
// M = strictly lower part of -(L11^-1) of the unit lower 64 x 64 block at
// (k0, k0), column-major in aux (2 words x 64 x 64)
int split_inv_l11(const double* A, int64_t lda, int64_t plane, int64_t k0, double* aux, cudaStream_t s);
// the L11 inverse area inside a split work buffer sized for order n
double* split_aux(char* ws, int64_t n);

// split-precision trailing update for DD (ozaki.cu): C -= L21 * U12
int split_update_dd(double* A, int64_t lda, int64_t plane, int64_t row0, int64_t m,
                    int64_t col0, int64_t N, int64_t k0, int nb, char* ws, size_t ws_bytes,
                    cudaStream_t s);
size_t split_workspace_bytes(int64_t n, int nb);
// work bytes of one split_product_dd with m rows and N columns
size_t split_product_bytes(int64_t m, int64_t N);
// work bytes of one LU of order n (lu_blocked): the header, and for the split
// update the trailing-update area plus a second product area that the
// look-ahead panel uses while the trailing update runs
size_t lu_workspace_bytes(int update, int64_t n);
// C -= L U (plus: C += L U) for one 64-wide slab of the inner dimension
int split_gemm_sub_dd(int64_t m, int64_t N, double* C, int64_t ldc, int64_t planeC, const double* L,
                      int64_t ldl, int64_t planeL, const double* U, int64_t ldu, int64_t planeU,
                      char* ws, size_t ws_bytes, cudaStream_t s, bool plus = false);
// the plain trailing update A22 -= L21 U12 in place (gemm_plain.cu): rows
// [row0, row0 + m) of columns [col0, col0 + N), inner columns [k0, k0 + nb)
template <int W>
int launch_gemm_plain(double* A, int64_t lda, int64_t plane, int64_t row0, int64_t m,
                      int64_t col0, int64_t N, int64_t k0, int nb, cudaStream_t s);
// C -= L U (add: C += L U) in plain multiword arithmetic, any K
template <int W>
int launch_gemm_plain_ptr(int64_t m, int64_t N, int K, double* C, int64_t ldc, int64_t planeC,
                          const double* L, int64_t ldl, int64_t planeL, const double* U, int64_t ldu,
                          int64_t planeU, cudaStream_t s, bool add = false);

// ---- batched blocked LU (batched.cu drives these per panel step) --------
// A batch in the packed layout: system s has order n[s], its matrix of w
// words at A + w*moff[s] with lda = n[s] and plane n[s]^2, its pivots at
// piv + voff[s].  `order` lists the systems largest first, so the systems
// still active at panel step k0 (n > k0) are order[0 .. act).
struct BatchView {
  const int* order;
  const int* n;
  const int64_t* moff;
  const int64_t* voff;
};

// one work item of a trailing update: system order[pos], tile (ti, tj)
struct TileEntry {
  int pos, ti, tj, pad;
};

constexpr int kBatchNb = 64;   // panel width of the batched blocked LU

// panel columns [k0 + c_off, k0 + c_off + width) of rows [k0 + c_off, n); the
// row swaps are applied inside those columns only
template <int W>
int launch_bpanel(const BatchView& bv, int act, int nmax, int k0, int c_off, int width, double* A, int64_t* piv,
                  int64_t* info, cudaStream_t s);
// row swaps k0 + [sw_lo, min(sw_hi, kb)) on the columns
// [max(0, k0 + c_lo), min(n, k0 + c_hi)); max_cols bounds the column count
template <int W>
int launch_bswap(const BatchView& bv, int act, int k0, int sw_lo, int sw_hi, int c_lo, int c_hi, int max_cols,
                 double* A, const int64_t* piv, cudaStream_t s);
// inside the panel, for the block of 2h columns at column offset c_off: the
// top h rows of its right half get the left half's swaps, then the unit
// lower h x h solve (h = 8, 16 or 32)
// batched: the plans of the panel swaps k0 + [sw_lo, min(sw_hi, kb)) of every
// active system (one warp each, plans[pos]), and their gather on the columns
// [max(0, k0 + c_lo), min(n, k0 + c_hi))
int launch_bswap_plan(const BatchView& bv, int act, int k0, int sw_lo, int sw_hi, const int64_t* piv,
                      SwapPlan* plans, cudaStream_t s);
template <int W>
int launch_bswap_apply(const BatchView& bv, int act, int k0, int c_lo, int c_hi, int max_cols, double* A,
                       const SwapPlan* plans, cudaStream_t s);
template <int W>
int launch_btrsm_sub(const BatchView& bv, int act, int k0, int c_off, int h, double* A, const int64_t* piv,
                     cudaStream_t s);
template <int W>
int launch_btrsm(const BatchView& bv, int act, int max_cblocks, int k0, double* A, const int64_t* piv,
                 cudaStream_t s);
template <int W>
int launch_bgemm_plain(const BatchView& bv, const TileEntry* tiles, int64_t ntiles, int k0, double* A,
                       cudaStream_t s);
// rows x columns of one plain-GEMM tile for W words
void gemm_plain_tile_shape(int W, int* bm, int* bn);

// split update of the batch (ozaki.cu): per active system with trailing
// order m = n - k0 - 64 > 0, C -= L21 U12 on the 128 x 16 tiles listed in
// `tiles`; `bases[pos]` = {first A-slice tile, first B-slice tile} of that
// system in the slice area; the slicing grids are act x max_mt (128-row
// tiles) and act x max_cb (128-column blocks).
constexpr int kSplitTileM = 128;
constexpr int kSplitTileN = 16;
// Operand geometries (ozaki.cu): the trailing update, and the TRSM as a
// product with the explicit inverse of L11 (aux: per active position, the
// strictly lower part of -(L11^-1), 2 words x 64 x 64, column-major).
constexpr int kGeomTrail = 0;
constexpr int kGeomTrsmInv = 1;
constexpr int kGeomPanelInner = 2;   // inside the panel: right half -= left half x solved top rows
                                     // (block of 2h columns at column offset c_off)
size_t split_batched_workspace_bytes(int64_t a_tiles, int64_t b_tiles);
int split_bupdate_dd(const BatchView& bv, int geom, int c_off, int h, int act, int max_mt, int max_cb,
                     const TileEntry* tiles,
                     int64_t ntiles, const int2* bases, int64_t a_tiles, int64_t b_tiles, int k0, double* A,
                     const double* aux, char* ws, size_t ws_bytes, DeviceStatus* status, cudaStream_t s);
// the two halves of split_bupdate_dd: the slices of every active system's
// operands, then the products of the tiles given (any subset of the step's
// tiles, in any order, once the slices are in place)
int split_bslice_dd(const BatchView& bv, int geom, int c_off, int h, int act, int max_mt, int max_cb,
                    const int2* bases, int64_t a_tiles, int64_t b_tiles, int k0, double* A, const double* aux,
                    char* ws, size_t ws_bytes, cudaStream_t s);
int split_bgemm_dd(const BatchView& bv, int geom, int c_off, int h, const TileEntry* tiles, int64_t ntiles,
                   const int2* bases, int64_t a_tiles, int64_t b_tiles, int k0, double* A, const double* aux,
                   char* ws, size_t ws_bytes, DeviceStatus* status, cudaStream_t s);
int split_binv_l11(const BatchView& bv, int act, int k0, const double* A, double* aux, cudaStream_t s);

// Strassen's recursion over the block matrix product (strassen.cu): C = A B,
// n x n, n divisible by 2^levels (split: DD and (n >> levels) % 64 == 0)
size_t strassen_workspace_bytes(int w, int update, int levels, int64_t n);
int strassen_run(int w, int update, int levels, int64_t n, const double* A, int64_t lda, const double* B,
                 int64_t ldb, double* C, int64_t ldc, char* ws, size_t ws_bytes, cudaStream_t s);

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
