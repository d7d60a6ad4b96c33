// Host-side model of the two-site problem: quantum-number bases, block-sparse
// operator tables, the NC term list and the sigma work list.
//
// Everything here is integer bookkeeping plus term coefficients; it runs once
// per operator skeleton (Sec. II.G (ii): the GEMM list is generated once per
// site and block-index lists once per skeleton). The floating-point work of
// the hot path runs in the CUDA kernels.
#pragma once

#include <cstdint>
#include <map>
#include <memory>
#include <utility>
#include <stdexcept>
#include <string>
#include <vector>

namespace dmrg {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// q = (N, 2Sz), ordered lexicographically.
struct QN {
  int n = 0, s = 0;
  bool operator<(const QN& o) const { return n < o.n || (n == o.n && s < o.s); }
  bool operator==(const QN& o) const { return n == o.n && s == o.s; }
  bool operator!=(const QN& o) const { return !(*this == o); }
  QN operator+(const QN& o) const { return {n + o.n, s + o.s}; }
  QN operator-(const QN& o) const { return {n - o.n, s - o.s}; }
  QN neg() const { return {-n, -s}; }
};

inline int spin_of(int p) { return (p % 2 == 0) ? 1 : -1; }

// Ascending list of sectors with dimensions and offsets.
struct Basis {
  std::vector<QN> q;
  std::vector<int> dim;
  std::vector<long long> off;
  long long total = 0;
  void finish();             // sort check + offsets
  int find(QN x) const;      // sector index or -1
  int size() const { return (int)q.size(); }
};

// One dense block of a stored operator: rows = dim(qout), cols = dim(qin),
// row-major at element offset `off` of the owning store.
struct OpBlock {
  int qin, qout;
  int rows, cols;
  long long off;
};

struct OpDesc {
  QN dq;
  int parity = 0;
  bool sym = false;
  std::vector<OpBlock> blocks;   // ascending qin
  std::vector<int> by_qin;       // sector index -> block index or -1
};

// Stored operators of one block, in canonical order. NC form: left kind H,
// a+_p (p<nL), R^L_p (nL<=p<n), A_pr (p<r<nL), B_pq (p<=q<nL); right kind H,
// a_p (p>=nL), R^R_p (p<nL), P_pr (p<r<nL), Q_pq (p<=q<nL). CN form (App. B,
// Eq. h-cn): the same one-index operators, and two-index pairs over the right
// modes [nL, n): P^L_pr, Q^L_pq on the left, A_pr, B_pq on the right. Both
// forms have 1 + n + np^2 ops, np = number of modes the pairs run over.
struct NCIndex {
  int nL = 0, n = 0;
  bool cn = false;
  int pb() const { return cn ? nL : 0; }       // first mode of the pair range
  int np() const { return cn ? n - nL : nL; }  // modes in the pair range
  int count() const { return 1 + n + np() * np(); }
  int H() const { return 0; }
  // left kind
  int cd(int p) const { return 1 + p; }
  int RL(int p) const { return 1 + nL + (p - nL); }
  // right kind
  int d(int p) const { return 1 + (p - nL); }
  int RR(int p) const { return 1 + (n - nL) + p; }
  // both kinds (p, q, r in the pair range)
  int pair_strict(int p, int r) const {
    p -= pb();
    r -= pb();
    return p * np() - p * (p + 1) / 2 + (r - p - 1);
  }
  int pair_le(int p, int q) const {
    p -= pb();
    q -= pb();
    return p * np() - p * (p - 1) / 2 + (q - p);
  }
  int A(int p, int r) const { return 1 + n + pair_strict(p, r); }  // A / P / P^L index
  int B(int p, int q) const { return 1 + n + np() * (np() - 1) / 2 + pair_le(p, q); }  // B / Q / Q^L index
};

struct OpSet {
  Basis basis;
  std::vector<OpDesc> ops;
  long long elements = 0;
};

// Build the block tables of the canonical left or right operator list (NC
// form, or CN form when cn) over `basis`, offsets starting at `base` (left
// ops first, then right ops, in one flat store for the synthetic problem).
void build_nc_opset(OpSet& out, const Basis& basis, int nL, int n, bool left, long long base, bool cn = false);
// Add one operator with shift dq over `basis` (blocks wherever both sectors exist).
void add_op(OpSet& set, QN dq, int parity, bool sym, long long& cursor);

struct Term {
  int opL, opR;     // -1 = identity
  bool tL, tR;      // use the transpose of the stored operator
  double coef;
  int parR;         // fermion parity of the right operator
};
std::vector<Term> nc_terms(int nL, int n);
// CN partition (App. B, Eq. h-cn in spin orbitals): H_L x 1, 1 x H_R, the NC
// one-index terms, P^L_pr x A_pr and its transpose (nL <= p < r), and
// Q^L_pq x B_pq (nL <= p, q), over CN-form operator sets.
std::vector<Term> cn_terms(int nL, int n);
// Sub-Hamiltonian rank of every term of nc_terms(nL, n) among n_ranks
// (Sec. II.B, Eqs. proc-def and proc-def-nc in spin-orbital indices): terms
// with one left index p go to p mod P; terms with a left pair p <= r to
// (r(r+1)/2 + p) mod P, so O_pr and O_rp always share a rank; H_L x 1 and
// 1 x H_R go to rank 0.
std::vector<int> nc_term_ranks(int nL, int n, int n_ranks);
// The same for cn_terms(nL, n) (Eq. proc-def-cn): the pair of a CN term is
// its right-block pair p <= r (the larger indices).
std::vector<int> cn_term_ranks(int nL, int n, int n_ranks);

// Sub-Hamiltonian `rank` of n_ranks of an NC middle-bond problem (Sec. II.B,
// Eqs. sum-h, sub-h, proc-def): the terms nc_term_ranks gives that rank,
// their positions in the full term list, and the operators they use. On
// return L and R keep only those operators' blocks (the others have none),
// laid out contiguously from offset 0 (left operators first); canon_off
// holds, per kept block in the new store order, its element offset in the
// full canonical store (where the synthetic generator's counters start).
struct Partition {
  std::vector<Term> terms;
  std::vector<int> term_ids;
  std::vector<long long> canon_off;
  long long elements = 0;
};
void partition_nc(OpSet& L, OpSet& R, int nL, int n, int rank, int n_ranks, Partition& out);

struct PsiBlock {
  int qL, qR;       // sector indices in the left / right basis
  int mL, mR;
  long long off;
};
std::vector<PsiBlock> psi_layout(const Basis& L, const Basis& R, QN Qtot, long long* size);

// One (term, input block) product feeding output block `out`.
struct Task {
  long long aoff;   // left operator block offset (elements), -1 = identity
  long long boff;   // right operator block offset, -1 = identity
  int in_blk;       // input psi block
  int flags;        // bit0: left block used transposed; bit1: right block transposed
  double scale;     // coefficient times fermion sign
};

// Work unit of one CTA: tasks [t_begin, t_end) (all with output block out),
// rows [r0, r0+nrows) x cols [c0, c0+ncols) of that block; partial result to
// scratch at `slot` (nrows x ncols, row-major).
struct Item {
  int out, r0, nrows, c0, ncols, t_begin, t_end, pad;
  long long slot;
};
// Output tile and the contiguous item range whose partials sum into it.
struct Group {
  int out, r0, nrows, c0, ncols, i_begin, i_end, pad;
};

// One class of the normal-to-complementary sums (Sec. III.A): operators of
// one shift, so one block structure of E elements; see launch_opcomb.
struct CombClass {
  long long y_off, c_off, E;
  int x_start, n_out, n_in;
  int tile_start;   // first tile of the class in the launch
  int tiles_e;      // tiles along E
  int pad;
};
constexpr int COMB_TM = 64, COMB_TN = 128;

// One small strided GEMM C = A B (see launch_bgemm): A(i, k) =
// A[a + (ta ? k * lda + i : i * lda + k)], B(k, j) = B[b + (tb ? j * ldb + k :
// k * ldb + j)], C[c + i * ldc + j], i < m, j < n, k < kk.
struct GJob {
  long long a, b, c;
  int m, n, kk;
  int lda, ldb, ldc;
  int ta, tb;
};

struct WorkList {
  std::vector<Task> tasks;        // grouped by output block
  std::vector<int> out_start;     // tasks of output block b: [out_start[b], out_start[b+1])
  std::vector<Item> items;        // grouped by output tile (contiguous per group)
  std::vector<Group> groups;
  std::vector<int> schedule;      // item indices, most expensive first
  long long scratch_elems = 0;
  double flops = 0;          // algorithmic (min order)
  double bytes_ops = 0;      // operator bytes read (FP64), each product reading its two blocks
  // host only, parallel to tasks: index of each task's left / right stored
  // block in store order (left operators' blocks, then right), -1 = identity
  std::vector<int> task_ablk, task_bblk;
};

struct TileShape {
  int tm;          // rows per tile
  int tn;          // max cols per tile
  double target;   // minimum cost per item
  double per_task = 16384.0;  // fixed latency term of one task in the item cost
};

void build_tasks(const std::vector<PsiBlock>& blocks, const OpSet& L, const OpSet& R,
                 const std::vector<Term>& terms, WorkList& wl);
// Split every output block into tm x tn tiles and each tile's task list into
// items of about max(ts.target, total / want_items) flops.
void build_items(const std::vector<PsiBlock>& blocks, WorkList& wl, const TileShape& ts,
                 int want_items, int n_out = -1);

}  // namespace dmrg

namespace dmrg {

// ------------------------------------------------------------------ tensor-core path
// Split operator store: every stored block S (r x c) is kept as three bf16
// slices S = hi + mid + lo, each in 8x8 "core-matrix" tiles: tile (i8, j8)
// holds rows 8*i8.., cols 8*j8.. as 8 rows of 8 contiguous elements (128 B),
// tiles ordered j8 fastest, the three slices of one tile position
// interleaved (384 B); padding elements are zero. The same tiles serve as a
// K-major operand (S as MN x K) or an MN-major one (S^T) of tcgen05.mma.
struct TcBlock {
  long long tile;   // first tile position of the block
  int R8, C8;       // tile rows / cols of the stored block
};

struct TcPsiBlock {
  long long tile;   // first tile position of the block in the psi split
  int R8, C8;       // rows padded to an even number of tile rows
  int m, n;
};

// Work of the tensor-core sigma. For one output tile (rows r0.. of at most
// 128, columns c0.. of at most 128) of output block b', the products of all
// terms that read the same psi block b with the same transposition flags
// form a class: sigma_b'[tile] += sum_t c_t L_t[rows, :] psi_b R_t[cols, :]^T.
// A unit is up to TC_MAX_G terms of one class whose left-operator rows are
// stacked in one 128-row operand, so one chain of MMAs gives X_t = L_t psi_b
// for all of them (stage 1); each term's X_t R_t^T then accumulates into the
// tile (stage 2). Stage 1 runs over 128-column chunks of psi; stage 2 over
// 64-column halves of each chunk. The FP32 tile accumulator is added into
// the item's running sum (FP32 pairs, about 48 bits) after every flush group
// of terms within one half (the launch bounds the main MMA steps of a
// group), which bounds the length of any FP32 accumulation chain.
constexpr int TC_MAX_G = 16;
enum { TC_TA = 1, TC_TB = 2, TC_ZERO = 4, TC_DONE = 8, TC_ITEM_FIRST = 16, TC_ITEM_LAST = 32 };
struct TcTermRec {          // 24 bytes
  long long a_tile, b_tile; // left / right operator blocks (identity blocks included)
  float scale;              // coefficient times fermion sign
  int pad;
};
struct TcUnitRec {          // 80-byte header + 16 terms = 464 bytes
  int flags;                // TC_TA (left used transposed), TC_TB (right transposed), TC_ZERO, TC_DONE,
                            // TC_ITEM_FIRST / TC_ITEM_LAST (first / last record of an item)
  int nterm;                // terms in the unit (<= TC_MAX_G)
  int tm, tn;               // rows / columns of the output tile
  int tm8;                  // row groups of one term in the stacked operand (ceil(tm / 8))
  int r0g, c0g;             // tile origin (row / column group) inside the output block
  int m, n;                 // psi block rows / columns
  int pblk;                 // psi block index
  short aR8, aC8, bR8, bC8; // stored tile geometry of the left / right blocks
  short pR8, pC8;           // psi tile geometry
  long long p_tile;         // psi tiles
  long long slot;           // the item's partial tile (tm x tn, row-major)
  int pad[2];
  TcTermRec t[TC_MAX_G];
};

// Output tile and its record range; same layout as Item (r_begin/r_end in
// the place of the task range) so the reduction can read it. kind 0: unit
// records of the tensor-core kernel; kind 1 / 2: small terms (SmallTerm) of the
// CUDA-core kernel.
struct TcItem {
  int out, r0, nrows, c0, ncols, r_begin, r_end, kind;
  long long slot;
};

// Classes whose blocks (output tile and psi block) are all at most
// TC_SMALL_MAX wide fill a tcgen05 instruction (128 x 16 x 16 at least) by a
// few percent; they run on the CUDA cores instead, in FP32 products of the
// operators (hi + mid + lo of their split, K <= 32 per product) with FP64
// sums over terms.
constexpr int TC_SMALL_MAX = 32;
// Small items whose blocks are all at most TC_SMALL_MID wide (kind 2) run
// with a smaller footprint than the rest of the small classes (kind 1).
constexpr int TC_SMALL_MID = 16;
struct SmallTerm {          // 32 bytes
  long long a_tile, b_tile; // first split tile of the left / right stored block, -1 = identity
  int in_blk;               // psi block
  int flags;                // bit0: left used transposed, bit1: right used transposed
  double scale;
};

// Allocator whose resize() leaves elements uninitialized (records are
// written in parallel, each by the thread that fills its item).
template <class T>
struct NoInit : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = NoInit<U>;
  };
  NoInit() = default;
  template <class U>
  NoInit(const NoInit<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};

struct TcPlan {
  std::vector<TcBlock> opblocks;        // tiles of every stored block, store order
  std::vector<TcBlock> identL, identR;  // identity blocks per sector of the left / right basis
  long long n_tiles = 0;                // tile positions of the operator split
  std::vector<TcPsiBlock> psi;
  long long psi_tiles = 0;
  std::vector<TcItem> items;            // grouped by output tile
  std::vector<int> schedule;            // kind-0 items, most expensive first
  std::vector<Group> groups;
  long long scratch_elems = 0;
  std::vector<TcUnitRec, NoInit<TcUnitRec>> recs;  // kind-0 item i: records [items[i].r_begin, items[i].r_end)
  std::vector<SmallTerm> small;         // kind-1/2 item i: terms [items[i].r_begin, items[i].r_end)
  // per record and term slot (record * TC_MAX_G + q): split-block indices of
  // the left and right blocks (stored blocks in store order, then the
  // identity blocks of the left and right sectors); -1 for unused slots
  std::vector<int> term_blk;
  std::vector<int> small_blk;           // per small term (2k, 2k+1): split-block indices as in term_blk
  std::vector<int> small_schedule;      // kind-2 items, then kind-1 items, each most expensive first
  int n_small_mid = 0;                  // kind-2 items (the head of small_schedule)
  long long n_terms = 0;                // term products (tasks x tiles), counted once
  long long n_units = 0;
  double mma_macs = 0;                  // multiply-adds issued per slice product (padding included)
};

struct TcShape {
  int want_items;           // items to split the work into (a multiple of the SM count)
  double unit_cost = 128.0 * 128 * 64;  // fixed cost of a unit in the item split, in multiply-adds
};
void build_tc_plan(const std::vector<PsiBlock>& blocks, const OpSet& L, const OpSet& R,
                   const WorkList& wl, TcPlan& plan, const TcShape& shape);

}  // namespace dmrg
