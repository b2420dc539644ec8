// Internal declarations shared by the TSQR / CAQR translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace tsqr {

// Bits of the device status word.
constexpr int kStatusNonfinite = 1;
constexpr int kStatusTimeout = 2;

// Threads per CTA of the factor and apply kernels.
constexpr int kLeafThreads64 = 128;  // FP64 leaves
constexpr int kLeafThreads32 = 256;  // FP32-storage leaves
constexpr int kLeafThreadsBig = 512; // leaves whose tile leaves room for one CTA per SM
constexpr int kNodeThreads = 128;
constexpr int kApplyThreads = 256;
// Columns of C handled by one CTA of the apply kernels.
constexpr int kApplyCols = 64;
// Rows of a leaf staged per pass in the apply kernels.
constexpr int kApplyRows = 32;
// Largest n the kernels are built for.
constexpr int kMaxN = 128;
// Leaf height cap of CAQR panels with FP32 storage (the BF16x3 update
// kernel takes any height), and the BF16x3 update's largest panel width.
constexpr int kBf16x3MaxLeaf = 512;
constexpr int kBf16x3MaxN = 64;

// Three apply modes: C <- Q^T C, C <- Q C, and "form": C <- Q [X; 0] where X
// is read from the first n rows of the block and the rest of the block is
// written without being read.
enum ApplyMode : int { kApplyQT = 0, kApplyQ = 1, kApplyForm = 2 };

// Leaf Householder QR of all row blocks of A (Section 2.1, Eq. TSQR_binarytree_1).
template <typename T>
struct LeafFactorArgs {
  T* A;             // m x n, column-major; leaf rows overwritten with Y and R_i
  int64_t lda;
  int64_t m;        // total rows
  int n;            // columns
  int64_t h;        // nominal leaf height; leaf i starts at row i*h
  int64_t nleaves;  // the last leaf runs to row m
  int ld_s;         // shared-memory leading dimension of the leaf tile (odd)
  T* R;             // nleaves x (n x n): leaf R factors, level-0 items of the tree
  T* tau;           // nleaves x n
  T* Tw;            // nleaves x (n x n): compact-WY T of each leaf
  int* status;
  // When set, the leaf rows are read from here (column stride ldsrc; for
  // example a mapped page-locked host matrix) and only written to A.
  const T* Asrc;
  int64_t ldsrc;
};

// Structured QR of up to q stacked triangles per node (Section 2.1,
// Eq. TSQR_binarytree_2): nodes of one tree level.
template <typename T>
struct NodeFactorArgs {
  const T* Rin;     // items of the level below: nin x (n x n), upper triangular
  int64_t nin;
  int arity;        // q
  int n;
  int64_t nodes;    // ceil(nin / q)
  T* Rout;          // nodes x (n x n)
  T* Y;             // nodes x (q-1) x (n x n): upper-triangular reflector blocks
  T* tau;           // nodes x n
  T* Tw;            // nodes x (n x n): compact-WY T
  int* status;
};

template <typename T>
struct LeafApplyArgs {
  const T* Y;       // the factored A: leaf Householder vectors
  int64_t ldy;
  int64_t m;
  int n;
  int64_t h;
  int64_t nleaves;
  const T* Tw;      // nleaves x (n x n)
  T* C;             // m x k
  int64_t ldc;
  int64_t k;
  int mode;         // ApplyMode
  // Set by the launcher: work units (leaf, 64-column chunk), leaf fastest,
  // one per CTA; units from split_from on are cut into `split` column
  // pieces (CTAs), so that the last, partial wave is made of short pieces.
  int64_t split_from;
  int split;
};

template <typename T>
struct NodeApplyArgs {
  const T* Y;       // nodes x (q-1) x (n x n)
  const T* Tw;      // nodes x (n x n)
  int64_t nin;      // items of the level below
  int arity;
  int n;
  int64_t nodes;
  int64_t slot_stride;  // rows between consecutive items of the level below
  T* C;
  int64_t ldc;
  int64_t k;
  int mode;
  // Set by the launcher: units (node, 64-column chunk), node fastest; units
  // from split_from on are cut into `split` column pieces.
  int64_t split_from;
  int split;
};

// Hybrid tree: chains of L consecutive leaves, each factored by one CTA as
// a flat tree (Section 2.1); chain c covers leaves [c L, min((c+1) L, nleaves)).
template <typename T>
struct ChainFactorArgs {
  T* A;             // m x n; leaf rows overwritten with their reflectors
  int64_t lda;
  int64_t m;
  int n;
  int64_t h;        // rows per leaf (the last leaf runs to m)
  int64_t nleaves;
  int64_t L;        // leaves per chain
  int64_t nchains;
  int ld_s;         // shared-memory leading dimension (odd, >= rows of a stacked tile)
  T* R;             // nchains x (n x n): the chains' R factors
  T* tau;           // nleaves x n
  T* Tw;            // nleaves x (n x n)
  int* status;
};

template <typename T>
struct ChainApplyArgs {
  const T* Y;       // the factored A
  int64_t ldy;
  int64_t m;
  int n;
  int64_t h;
  int64_t nleaves;
  int64_t L;
  int64_t nchains;
  const T* Tw;      // nleaves x (n x n)
  T* C;             // m x k
  int64_t ldc;
  int64_t k;
  int mode;         // ApplyMode
};

template <typename T>
cudaError_t launch_chain_factor(const ChainFactorArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_chain_apply(const ChainApplyArgs<T>& a, cudaStream_t s);
size_t chain_apply_smem(int n, size_t elem);
int chain_factor_resident(int n, int ld, size_t elem);

template <typename T>
cudaError_t launch_leaf_factor(const LeafFactorArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_node_factor(const NodeFactorArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_leaf_apply(const LeafApplyArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_node_apply(const NodeApplyArgs<T>& a, cudaStream_t s);

// C <- C - Y T^T Y^T C per leaf with three split products on tcgen05 (FP32
// storage, n <= 64): BF16 terms (kind::f16) or, with tf32, TF32 terms.
cudaError_t launch_leaf_update_split3(const LeafApplyArgs<float>& a, bool tf32, int* status, cudaStream_t s);

// d = sign(diag Rroot) (sign(0) = +1); Rout = D * triu(Rroot), ldr.  Entries
// below the diagonal of Rout are zeroed when zero_lower, left alone otherwise.
template <typename T>
cudaError_t launch_sign_fix(const T* Rroot, int n, T* d, T* Rout, int64_t ldr, bool zero_lower, cudaStream_t s);
// Rows 0..n-1 of C (k columns) scaled by d.
template <typename T>
cudaError_t launch_scale_rows(T* C, int64_t ldc, int n, int64_t k, const T* d, cudaStream_t s);
// Q(0:n, 0:n) = diag(d) (the identity when d is null).
template <typename T>
cudaError_t launch_init_form(T* Q, int64_t ldq, int n, const T* d, cudaStream_t s);
// Q(0:n, 0:k) = diag(d) X (d may be null).
template <typename T>
cudaError_t launch_init_form_mul(T* Q, int64_t ldq, int n, int64_t k, const T* d, const T* X, int64_t ldx,
                                 cudaStream_t s);
// Copy the n x n upper triangle of src (ld n) into dst (ldd), zero below.
template <typename T>
cudaError_t launch_copy_upper(const T* src, int n, T* dst, int64_t ldd, cudaStream_t s);

// X = R^{-1} B for upper-triangular R (n <= kMaxN); B may alias X.  A zero or
// non-finite diagonal entry sets kStatusNonfinite in *status (if non-null).
template <typename T>
cudaError_t launch_solve_upper(int n, int64_t k, const T* R, int64_t ldr, const T* B, int64_t ldb, T* X, int64_t ldx,
                               int* status, cudaStream_t s);
// out[j] = ||B(r0:m, j)||_2 (FP64 sums of squares in acc, k doubles).
template <typename T>
cudaError_t launch_column_norms(int64_t r0, int64_t m, int64_t k, const T* B, int64_t ldb, double* acc, T* out,
                                cudaStream_t s);

// Shared-memory bytes the leaf factor kernel needs for a leaf of hmax rows.
size_t leaf_factor_smem(int n, int hmax, size_t elem);
int leaf_factor_ld(int hmax);

}  // namespace tsqr
