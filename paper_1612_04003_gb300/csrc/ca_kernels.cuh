// ca_kernels.cuh -- declarations of the CA-BCD / CA-BDCD device kernels.
#pragma once
#include "ca_common.cuh"

__global__ void k_sample(unsigned long long seed, long long h0, long long H, int b, long long N,
                         int* out);

// Host launchers of the templated kernels (defined in ca_kernels.cu; the
// templates are launched only from their own translation unit).
void launch_gram_simt(bool f64, dim3 grid, cudaStream_t st, const void* A, long long lda,
                      long long N, long long K, const int* idx, int sb, const double* v,
                      long long chunks_per_split, int sbp, double* part, double* ppart,
                      unsigned* err);
// a4: reduce the split-K partials (with ndiag > 0 also inverting the diagonal
// blocks, b <= 16), invert them separately (launch_factor, from R), then the
// chain (fast form) or the general solve.
void launch_reduce(bool f32_partials, int grid, size_t smem, cudaStream_t st, const void* part,
                   const double* ppart, int P, int sbp, double* R, float2* Rs, double* pvec,
                   float2* Ginv, int ndiag, const SolveArgs& sa, unsigned* err);
void launch_chain(int b, size_t smem, cudaStream_t st, const float2* Rs, const double* pvec,
                  const float2* Ginv, const SolveArgs& sa, unsigned* err);
void launch_factor(cudaStream_t st, const double* R, const SolveArgs& sa, float2* Ginv,
                   unsigned* err);
// a4 in one programmatic-dependent launch (FP32 partials, b <= 16): reduce
// with the diagonal-block inverses (ndiag = s_cur CTAs), then the chain on the
// CTA that finishes last.  Returns a cudaError_t.
int launch_reduce_chain(int grid, size_t smem, cudaStream_t st, const float* part,
                        const double* ppart, int P, int sbp, double* R, float2* Rs, double* pvec,
                        float2* Ginv, int ndiag, const SolveArgs& sa, unsigned* err,
                        unsigned* ticket);
__global__ void k_factor(const double* R, SolveArgs sa, float2* Ginv, unsigned* err);
#define CA_FAST_B 32
#define CA_FAST_SB 256
// panel: FP32 A stored as 32-column panels [K/32][N][32] (k_pack_panels).
void launch_update_dense(bool f64, unsigned grid, size_t smem, cudaStream_t st, const void* A,
                         long long lda, long long N, long long K, const int* idx, int sb,
                         const double* delta, double cU, double* v, float2* v2, unsigned* err,
                         bool panel);
void launch_recompute_dense(bool f64, dim3 grid, cudaStream_t st, const void* A, long long lda,
                            long long N, long long K, const double* x, const float2* x2, double c1,
                            long long rows_per_split, double* v, bool panel,
                            const unsigned* nz = nullptr);
__global__ void k_pack_panels(const float* A, long long N, long long K, long long lda, float* Pn);
int set_solve_smem_limit(int bytes);

__global__ void k_solve(const double* R, const double* pvec, SolveArgs sa, unsigned* err);

__global__ void k_axpby_init(const double* y0, double c0, long long K, double* v, unsigned* nz);
__global__ void k_nonzero(const double* x, long long N, float2* x2, unsigned* nz);
__global__ void k_split(const double* v, long long K, long long Kpad, float2* v2);

__global__ void k_scatter_csr(const long long* rowptr, const int* col, const float* val,
                              const int* idx, long long nrows_total, long long ncols,
                              long long nlist, const double* coef, double c, double* v,
                              unsigned* err);

__global__ void k_selftest_wait(unsigned long long limit_ns, unsigned* err);
__global__ void k_symmetrize(const double* R, int ldr, int sb, double* G);

// tcgen05 Gram (ca_gram_tc.cu): host-side launcher.  Returns a cudaError_t.
// Computes FP32 partials part[c][j][i] (c < P, stride sbp; stored transposed) of
// sum_{k in split c} Y[i][k] Y[j][k] for the tiles covering j <= i, and FP64
// partials ppart[c][i] of sum_k Y[i][k] v[k], v given as FP32 pairs
// (hi, lo) zero-padded to a multiple of 32 entries.  sbp (the tile height and
// the row stride of the partials) is 32, 64, 128 or 256 >= sb.
// Fused deferred update of the previous outer step (see ca_gram_tc.cu).
struct GramUpdate {
  const int* idx;       // rows of the previous outer step (sb of them); sb = 0: none
  int sb;
  const double* delta;  // their Delta
  double cU;            // v -= cU * Yprev^T Delta
  float2* v2;           // K entries as FP32 (hi, lo) pairs: read, updated in place
  const float* rscale;  // scaled FP16 Gram: power-of-two multiplier of each row of A
  // true only when the preceding grid in the stream writes none of A, the
  // sampled indices, v2 or rscale (the reduce + chain launch of the solves):
  // the CTAs then read them and start their loads before waiting for that
  // grid; otherwise they wait first
  bool early;
};

// A shared Gram launch over several problems (the batched solves): problem
// descriptors, the units of work (atoms [a0, a1) of one problem into one of
// its split-K partial slots) and each CTA's range of units.
struct GramInst {
  const float* A;       // the problem's A in 32-column panels
  long long lda, N, K;
  const int* idx;       // sampled rows of its current outer step
  int sb;
  const float2* v2;     // FP32 pairs of its projection vector (updated in place)
  float* part;          // its partial slots: nslots x SBP x SBP
  double* ppart;        // nslots x SBP
  GramUpdate u;         // its pending deferred update (u.sb = 0: none; u.v2 = v2)
};
struct GramUnit {
  int inst, slot;
  long long a0, a1;
};
struct GramBatchArgs {
  const GramInst* insts;
  const GramUnit* units;
  const int* unit_begin;  // units of CTA c: unit_begin[c] .. unit_begin[c+1]-1
  bool early;             // as GramUpdate::early, for the whole launch
};
// Consecutive outer steps k0 .. k0+npass-1 of one dense solve (FP32 A in
// 32-column panels, BF16x3 or scaled-FP16 Gram, s*b <= 128, b <= 8) in one
// persistent cooperative launch of Pg Gram CTAs + 1 chain CTA (ca_persist.cu).
struct PersistArgs {
  const float* A;        // panels [K/32][N][32], zero-padded past K
  long long N, K, natoms;
  const int* idx_all;    // sampled indices: step k at idx_all + k * sb
  int sb;                // s * b of every step of the launch
  long long k0;
  int npass;
  int na;                // region-A atoms of each Gram CTA: 0, or more than the load-ring
                         // depth (persist_load_ring), as natoms / Pg must be
  const int* prev_idx;   // rows of step k0 - 1 (prev_sb = 0: none)
  int prev_sb;
  double* delta2[2];     // Delta of step k in delta2[k & 1]
  float2* v2;            // FP32 pairs of v (K entries, zero-padded to a multiple of 32)
  double cU;
  const float* rscale;   // scaled FP16: power-of-two multiplier of each row of A
  float* part;           // Pg x sbp x sbp FP32 Gram partials (transposed)
  double* ppart;         // Pg x sbp projection partials
  double* R;
  float2* Rs;
  double* pvec;
  float2* Ginv;
  SolveArgs sa;          // solve constants (idx and delta are set per step)
  unsigned* cnt;         // 3 counts, zero on entry
  size_t chain_smem;     // shared memory of the chain (<= the Gram CTAs')
};
// mode: 2 = BF16x3, 3 = scaled FP16; grid = Pg + 1 <= number of SMs.
// Returns a cudaError_t.
int launch_persist(const PersistArgs& a, int grid, int sbp, int mode, unsigned* err,
                   cudaStream_t stream);
// Depth of the persistent kernel's load ring (stages in flight per CTA).
int persist_load_ring(int sbp, int mode);

// Shared launch of P CTAs; sbp = 32, 64 or 128 (>= every problem's s*b).
int launch_gram_tc_batch(const GramBatchArgs& bt, int P, int sbp, int three_pass, unsigned* err,
                         cudaStream_t stream);

// a4 of a shared launch: per problem its partial slots, reduction targets,
// solve arguments and the number of reducing CTAs (>= ndiag + 1); role of a
// CTA of the reduce grid: problem and index among that problem's CTAs.
struct RedInst {
  const float* part;
  const double* ppart;
  int P, sbp, ndiag;
  double* R;
  float2* Rs;
  double* pvec;
  float2* Ginv;
  SolveArgs sa;
};
struct RedRole {
  int inst, cta, ncta;
};
int launch_reduce_batch(int grid, cudaStream_t st, const RedInst* insts, const RedRole* roles,
                        unsigned* err);
// one chain CTA per problem (b <= bmax <= 16, s*b <= 256)
int launch_chain_batch(int count, int bmax, size_t smem, cudaStream_t st, const RedInst* insts,
                       unsigned* err);

// Sparse dual, steps a2+a3 of one outer step from the CSR of X^T (row hash
// tables, ca_kernels.cu): G (ldr x ldr, transposed lower triangle, the one
// "partial" of the reduction) and the projections pvec[r] = x_{I_r}^T w, in
// one programmatic-dependent launch.  Then a4 by the reduction of that
// single FP64 partial, the diagonal inverses and the chain in one launch
// (b <= 16), and a5 by the scatter (programmatic dependent).
struct ca_csr_dev;
// Dense-sparse split of the sparse Gram: heavy features (columns of X^T in
// at least a quarter of the rows, CA_CSR_DENSE_MAX at most) get a column of
// the dense nrows x fd matrix Xd.  launch_csr_prepare: fill = false counts
// each column's entries into cnt (zero on entry); fill = true scatters the
// mapped entries into Xd (zero on entry; fd, the row length of Xd, a
// multiple of 8 with the columns past the mapped ones left zero).  The split
// Gram of a step: the
// Gram of the sampled rows of Xd (k_dgram, writes the strict lower
// triangle), then the remaining features' pair products (k_sgram, FP64
// atomics); sb <= 4096.
#define CA_CSR_DENSE_MAX 512
void launch_csr_prepare(cudaStream_t st, int num_sms, const ca_csr_dev& csr, long long nrows,
                        long long ncols, long long nnz, int* cnt, const int* dmap, int fd,
                        float* Xd, bool fill);
// The diagonal and projections of the sampled rows (k_csr_rows), and the
// strict lower triangle of their Gram: the split (k_dgram + k_sgram) or,
// split = false, one warp per pair (k_csr_gram_pairs, sb <= 128).
void launch_csr_rows(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                     long long ncols, int sb, int ldr, const double* w, double* G, double* pvec,
                     unsigned* err);
void launch_csr_offdiag(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                        long long ncols, int sb, int ldr, double* G, const int* dmap,
                        const float* Xd, int fd, bool split, const int* roff);
// Where each feature range of the split's sparse part starts in every row
// (csr_rangeoff_bytes of int offsets, formed once per solve; roff = nullptr
// in launch_csr_offdiag makes it search instead).
size_t csr_rangeoff_bytes(long long nrows, long long ncols);
void launch_csr_rangeoff(cudaStream_t st, const ca_csr_dev& csr, long long nrows, long long ncols,
                         int* roff);
// The fast a4 of the sparse dual (b <= 16) in two parts: launch_csr_prep
// (needs neither w nor alpha: diagonal-block inverses into Ginv and the
// cG-scaled FP32 pairs Rs of G's strict lower triangle; the diagonal from the
// row norms rn of launch_csr_rownorm, formed once per solve) and
// launch_csr_proj (the projections x_{I_p}^T w into pvec), both for the sa.sb
// sampled rows sa.idx; then the chain (launch_chain).
void launch_csr_rownorm(cudaStream_t st, const ca_csr_dev& csr, long long nrows, double* rn);
void launch_csr_prep(cudaStream_t st, int num_sms, const double* rn, long long nrows,
                     const double* G, const SolveArgs& sa, float2* Rs, float2* Ginv,
                     unsigned* err);
void launch_csr_proj(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                     long long ncols, int sb, const double* w, double* pvec, unsigned* err);
void launch_csr_gram(cudaStream_t st, int num_sms, const ca_csr_dev& csr, const int* idx,
                     long long nrows, long long ncols, int sb, int ldr, const double* w, double* G,
                     double* pvec, unsigned* err);
int launch_reduce_chain_f64(int grid, size_t smem, cudaStream_t st, const double* part,
                            const double* ppart, int sbp, double* R, float2* Rs, double* pvec,
                            float2* Ginv, int ndiag, const SolveArgs& sa, unsigned* err,
                            unsigned* ticket);
void launch_scatter_csr(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                        long long ncols, long long nlist, const double* coef, double c, double* v,
                        unsigned* err);

// Stopping criterion: *out += ||cP A v - cI x - cY y||^2 over the N rows of
// A (dense: row-major FP64 / FP32 or FP32 panels, v2 the FP32 split of v for
// FP32 A; csr: rows of the CSR matrix, FP64 v).  q: N doubles, zero on entry
// and on return.  *out must be zeroed by the caller.
struct ca_csr_dev {
  const long long* rowptr;
  const int* col;
  const float* val;
};
void launch_residual(cudaStream_t st, int num_sms, const void* A, bool f64, bool panel,
                     long long lda, long long N, long long K, const double* v, const float2* v2,
                     const ca_csr_dev* csr, double* q, const double* x, const double* y,
                     double cP, double cI, double cY, double* out);
// *out += sum_{r < len} (cx x[r] + cy y[r])^2 (y may be null), by the
// residual's reduction kernel with cP = 0; q must hold len zeros (they are
// written back as zeros).
void launch_sumsq(cudaStream_t st, int num_sms, double* q, const double* x, const double* y,
                  long long len, double cx, double cy, double* out);

// Scaled FP16 Gram: per-row power-of-two multipliers of A (k_row_scale).
void launch_row_scale(cudaStream_t st, const float* A, long long lda, long long N, long long K,
                      bool panel, float* rscale);

// panel: A is stored as 32-column panels (k_pack_panels), else row-major with
// leading dimension lda (16-byte aligned rows).  The fused update needs panels.
int launch_gram_tc(const float* A, long long lda, long long N, long long K, const int* idx, int sb,
                   const float2* v2, int P, int sbp, float* part, double* ppart, unsigned* err,
                   int three_pass, cudaStream_t stream, const GramUpdate* upd = nullptr,
                   bool panel = false);
int gram_tc_max_sb();
