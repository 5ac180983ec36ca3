// Internal declarations of the SP2 library: device data layout and kernel
// launchers.  Everything here is private to the shared library; the public
// boundary is include/sp2.h.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include "sp2.h"

namespace sp2 {

constexpr int TB = 32;          // tile edge (Section 6: small block size 32)
constexpr int TE = TB * TB;     // elements per tile

// A set of upper-triangle tiles (I <= J), sorted by (I, J).  Tile t's values
// live in a value pool at pool[slot[t] * TE .. + TE), row-major.
struct TileSet {
  int64_t nnzb = 0;
  int32_t* brow = nullptr;
  int32_t* bcol = nullptr;
  int32_t* slot = nullptr;
  int32_t* rowptr = nullptr;    // [nb + 1] offsets of each tile row
};

// Both-triangle view of a symmetric tile pattern, used by the products.
//  bits:  nb x words bitmap, bit K of row R set iff tile (R, K) or (K, R) is stored.
//  rowptr/col/ref: for row R, the stored neighbours K in ascending order; ref =
//  slot | (1u << 31) when X_RK is the transpose of the stored tile (K, R).
struct FullPattern {
  int32_t words = 0;
  uint32_t* bits = nullptr;
  int32_t* rowptr = nullptr;    // [nb + 1]
  int32_t* col = nullptr;       // [nnz]
  uint32_t* ref = nullptr;      // [nnz]
  int64_t nnz = 0;
};

constexpr uint32_t REF_T = 0x80000000u;

// Host-side count of the kernels this library has launched (reported per run).
extern thread_local long long g_launches;   // launches issued by this host thread

// Per-output-tile partial sums written by the fused epilogue.
struct Partials {
  double* e2 = nullptr;       // w * ||X~_IJ - S_IJ||_F^2  (w = 2 off the diagonal)
  double* trS = nullptr;      // trace part of S on diagonal tiles
  double* trX = nullptr;      // trace part of X~ on diagonal tiles
  double* n2 = nullptr;       // ||X_new tile||_F^2
  int32_t* ktiles = nullptr;  // number of K tiles that contributed
};

// Scalars of one fused step, reduced in a fixed order.
struct StepScalars {
  double e2, trS, trX, pad;
  long long triplets;
  long long pad2[3];
};

// ---------------------------------------------------------------- launchers
// pattern.cu
cudaError_t launch_bitmap(const TileSet& s, int nb, FullPattern& fp, cudaStream_t st);
cudaError_t launch_row_popc(const uint32_t* bits, int nb, int words, int32_t* counts, cudaStream_t st);
cudaError_t launch_scan_i32(const int32_t* in, int32_t* out_excl, int64_t n, int32_t* total_dev,
                            void* tmp, cudaStream_t st);
size_t scan_tmp_bytes(int64_t n);
cudaError_t launch_fill_full(const TileSet& s, int nb, FullPattern& fp, cudaStream_t st);
// out row I = a's row I | OR over K in a's row I of b's row K | {I}; upper:
// only J >= I (symmetric storage), else the whole row (general storage)
cudaError_t launch_product_bits(const FullPattern& a, const FullPattern& b, int nb, uint32_t* out_bits,
                                cudaStream_t st, bool upper = true);
cudaError_t launch_fill_upper_from_bits(const uint32_t* bits, int nb, int words, const int32_t* rowptr,
                                        int32_t* brow, int32_t* bcol, int32_t* slot, cudaStream_t st);
cudaError_t launch_rowptr_from_brow(const int32_t* brow, int64_t nnzb, int nb, int32_t* rowptr,
                                    cudaStream_t st);
cudaError_t launch_check_pattern(const int32_t* brow, const int32_t* bcol, int64_t nnzb, int nb,
                                 const double* val, int64_t n, int32_t* flag, cudaStream_t st);

// init.cu
cudaError_t launch_gershgorin(const FullPattern& fp, const double* pool, int nb, int64_t n, double* rowlo,
                              double* rowhi, cudaStream_t st);
cudaError_t launch_minmax(const double* lo, const double* hi, int64_t n, double* out2, cudaStream_t st);
cudaError_t launch_x0(const TileSet& f, const double* fpool, double* xpool, int64_t n, double lmax, double w,
                      double* n2, cudaStream_t st);

// square_f64.cu: X_new = c0 I + c1 Z + c2 * (A B  [+ B A])  on the tiles of `out`
struct SquareArgs {
  const FullPattern* A;  const double* apool;
  const FullPattern* B;  const double* bpool;   // B == A for the forward square
  bool sym_sum;                                 // add B A too (adjoint)
  const FullPattern* Z;  const double* zpool;   // tile (I, J) of Z (may be absent -> 0)
  const TileSet* out; double* outpool;
  double c0, c1, c2;
  int64_t n; int nb;
  Partials part;
  bool general = false;                         // both triangles stored: every tile has weight 1 in e^2
};
cudaError_t launch_square_f64(const SquareArgs& a, cudaStream_t st);
size_t reduce_work_bytes();
cudaError_t launch_reduce_step(const Partials& p, int64_t ntiles, StepScalars* out, void* work, cudaStream_t st);

// trunc.cu: choose the tiles to drop (Frobenius / Frob-Inf readings)
struct TruncWork;
size_t trunc_work_bytes(int64_t nnzb, int nb, int64_t part_tiles);
cudaError_t launch_truncate(const TileSet& x, const double* n2, int nb, double tau, int mode, int64_t part_tiles,
                            void* work, int32_t* keep, cudaStream_t st);

cudaError_t launch_tile_norms(const double* val, int64_t nnzb, double* n2, cudaStream_t st);

// Mixed-norm selection (Section 3, ||.||_m on a partition of part_tiles tiles):
// work of mixed_work_bytes(nnzb, nsb); synchronises the stream (one host round
// trip per bisection probe).
constexpr int MIXED_MAX_BLOCKS = 512;
size_t mixed_work_bytes(int64_t nnzb, int nsb);
double mixed_norm_bound_host(const unsigned long long* B2, int nsb);
cudaError_t mixed_select(const TileSet& x, const double* n2, int nb, double tau, int64_t part_tiles, void* work,
                         int32_t* keep, cudaStream_t st);

// compact.cu
cudaError_t launch_compact(const TileSet& in, const int32_t* keep, int nb, TileSet& out, int32_t* count_dev,
                           void* scan_tmp, int32_t* scan_buf, cudaStream_t st);
cudaError_t launch_gather_tiles(const TileSet& s, const double* pool, double* dst, cudaStream_t st);
cudaError_t launch_copy_index(const TileSet& s, int32_t* brow, int32_t* bcol, cudaStream_t st);
// dst tiles := scale * the tile of `src` at the same (I, J), 0 when absent; src
// needs rowptr; sym_diag symmetrises diagonal tiles.
cudaError_t launch_place(const TileSet& src, const double* spool, const TileSet& dst, double* dpool, double scale,
                         int sym_diag, cudaStream_t st);
cudaError_t launch_iota(int32_t* p, int64_t n, cudaStream_t st);
// *out = trace of the kept diagonal tiles of s (s needs rowptr; keep may be nullptr)
cudaError_t launch_trace_kept(const TileSet& s, const int32_t* keep, const double* pool, int nb, int64_t n,
                              double* out, cudaStream_t st);

// dense.cu: dense row-major matrix <-> upper tiles
// flag[I * nb + J] = 1 for every diagonal tile and every nonzero tile with J > I
cudaError_t launch_dense_tile_flags(const double* F, int64_t n, int64_t ld, int nb, int32_t* flag, cudaStream_t st);
cudaError_t launch_dense_tile_fill(const double* F, int64_t n, int64_t ld, int nb, const int32_t* flag,
                                   const int32_t* pos, int32_t* brow, int32_t* bcol, double* pool, cudaStream_t st);
// out := the symmetric matrix of the upper tiles (zero elsewhere), leading dimension ld
cudaError_t launch_tiles_to_dense(const int32_t* brow, const int32_t* bcol, const double* val, int64_t nnzb,
                                  int64_t n, int64_t ld, double* out, cudaStream_t st);

// general.cu: general (both-triangle) storage of the iterates
cudaError_t launch_bits_general(const TileSet& s, int nb, int words, uint32_t* bits, cudaStream_t st);
// CSC view of a general set with a symmetric pattern: ref[t] = slot (or index) of the mirror of t | REF_T
cudaError_t launch_csc_refs(const TileSet& s, const int32_t* slot, uint32_t* ref, cudaStream_t st);
// general set (entries of fp, values transposed where ref has REF_T) from a symmetric set's pool
cudaError_t launch_expand_general(const FullPattern& fp, int nb, const double* src, int32_t* brow, int32_t* bcol,
                                  double* dst, cudaStream_t st);
cudaError_t launch_upper_flags(const TileSet& s, int32_t* flag, cudaStream_t st);
cudaError_t launch_general_keep(const TileSet& s, const int32_t* posU, const int32_t* keepU, int32_t* keep,
                                cudaStream_t st);

// square_tc.cu: tcgen05 FP16-slice product (see the file header).  An
// operand is stored as panel records: for each super-row R (tile rows
// 4R..4R+3) and K tile present in its super-row bitmap, a header byte and the
// k FP16 slices of the 4 tiles (see k_panel_slices); Z's values are found
// through zslot.
struct TcOp {
  const uint32_t* sbits = nullptr;   // super-row bitmaps [nsr][words]
  const int32_t* spos = nullptr;     // index of the first record of each (R, word) [nsr][words]
  const uint8_t* head = nullptr;     // record headers
  const void* data = nullptr;        // record slices, k * 8 KB each
};
struct TcLaunch {
  TcOp P, Q;                 // S = sum_K P_IK Q_KJ (+ Q_IK P_KJ when two_pass)
  bool two_pass;
  double scale;              // product of the slice scales of P and Q (powers of two)
  const FullPattern* Z;      // the c1 term's matrix (values: zpool)
  const int32_t* zslot;      // value slot of each tile index of Z's pattern (nullptr: identity)
  const double* zpool;
  const uint32_t* obits;     // output pattern bitmap (upper tiles only)
  const int32_t* orowptr;
  const int32_t* list;       // active super-tiles
  const int32_t* count;      // their number on the device
  int32_t* work;             // work counter of the persistent kernel (zeroed by the caller)
  int64_t nsuper;            // grid size (one CTA per SM, capped by the upper bound)
  double* opool;
  Partials part;
  double c0, c1, c2;
  int64_t n;
  int nb, nsr, k, words;
  int32_t* err;
  void* scratch;             // nsuper * tc_tile_slots() * 128 * 128 int64 (epilogue staging per CTA)
  int seg_min;               // K loops of at least this many steps are accumulated in segments (0: never)
  int seg_ksteps = 16;       // K steps per segment (8 or 16)
  unsigned long long wait_ns = 2000000000ull;   // limit of every bounded wait in the kernel
  bool selftest = false;     // wait first on a barrier nothing arrives at (tests the timeout path)
  bool general = false;      // general storage: every output tile of the square, weight 1 in e^2
  bool split_supply = false; // B operand units through copy warps (cp.async) beside the bulk copies of A
  const double* dsq = nullptr;   // S_ii per global row in FP64 (symmetric square: the squared row norms)
  int glo = 0, ghi = -1;     // slice-pair groups s + t of the launch (ghi < 0: all, k - 1; at most 4 groups)
  int emode = 0;             // 0 full epilogue, 1 store S only, 2 full epilogue on S + the stored S
};
size_t panel_record_bytes(int k);
// dsq[i] = sum_k x_ik^2 from the per-record squared row sums rsq of an
// operand's panel records (spos: the operand's record offsets, nsr x words + 1)
cudaError_t launch_row_sq_sum(const int32_t* spos, int nsr, int words, const double* rsq, int64_t n, double* dsq,
                              cudaStream_t st);
int tc_tile_slots();   // tiles in flight between the producer and the epilogue of k_square_tc
// report_range: also report an out-of-range element (error bit 4) without one
// being present (self-test of the error path); rsq (nullptr: skipped): 128
// squared row sums per record, FP64, unscaled
cudaError_t launch_panel_slices(const uint32_t* index, int64_t nrec, const int32_t* slot, const double* pool,
                                void* data, uint8_t* head, int k, int32_t* err, double* rsq, double scale,
                                bool report_range, cudaStream_t st);
cudaError_t launch_popc_words(const uint32_t* bits, int64_t n, int32_t* cnt, cudaStream_t st);
cudaError_t launch_panel_fill(const FullPattern& fp, int nb, const uint32_t* sbits, const int32_t* spos,
                              uint32_t* index, cudaStream_t st);
cudaError_t launch_absmax(const TileSet& x, const double* pool, unsigned long long* out, cudaStream_t st);
cudaError_t launch_upper_bits(const TileSet& x, int nb, int words, uint32_t* bits, cudaStream_t st);
cudaError_t launch_super_bits(const FullPattern& fp, int nb, int nsr, uint32_t* sb, cudaStream_t st);
int64_t super_order_size(int nsr);   // length of the (padded) launch-order index space
cudaError_t launch_super_flags(const uint32_t* obits, int nb, int words, int nsr, int32_t* flag, cudaStream_t st,
                               bool general = false);
cudaError_t launch_super_fill(const int32_t* flag, const int32_t* pos, int64_t n, int nsr, int32_t* list,
                              cudaStream_t st);
cudaError_t launch_square_tc(const TcLaunch& L, cudaStream_t st);

}  // namespace sp2
