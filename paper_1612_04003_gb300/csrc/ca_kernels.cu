// ca_kernels.cu -- CUDA-core kernels of the CA-BCD / CA-BDCD outer step (sm_103a).
//
// Generic form used by every kernel here: A is an N x K row-major matrix whose
// rows are sampled (primal: A = X, N = d, K = n; dual: A = X^T, N = n, K = d),
// Y = the s'*b sampled rows of A, v the K-vector the Gram pass projects on
// (primal: rho = y - z with z = X^T w; dual: w).
#include <algorithm>
#include <type_traits>

#include "ca_kernels.cuh"
#include "ca_solve.cuh"

// ---------------------------------------------------------------------------
// a1: sampling.  One warp per block h: Floyd's algorithm over [0, N), the
// membership test spread over the lanes.  Alg. 1-4 "choose ... uniformly at
// random without replacement".
// ---------------------------------------------------------------------------
__global__ void k_sample(unsigned long long seed, long long h0, long long H, int b, long long N,
                         int* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long hl = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (hl >= H) return;
  const unsigned long long h = (unsigned long long)(h0 + hl);
  int* blk = out + hl * (long long)b;
  uint64_t words[4] = {0, 0, 0, 0};
  for (int m = 0; m < b; ++m) {
    if ((m & 3) == 0) {
      uint64_t x[4] = {h, (uint64_t)(m >> 2), 0ull, 0ull};
      ca_philox4x64_10(x, Philox4x64Key{seed, 0ull});
      words[0] = x[0]; words[1] = x[1]; words[2] = x[2]; words[3] = x[3];
    }
    const uint64_t u = words[m & 3];
    const long long J = N - b + m;
    const long long t = (long long)__umul64hi(u, (uint64_t)(J + 1));
    bool hit = false;
    for (int q = lane; q < m; q += 32) hit |= (blk[q] == t);
    const bool seen = __any_sync(0xffffffffu, hit);
    if (lane == 0) blk[m] = (int)(seen ? J : t);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// a2+a3 on CUDA cores in FP64: Gram partials of the sampled rows and their
// projection on v, split over K.  Grid (P, tile pairs): CTA (c, t) computes
// the 64x64 tile (I, J), I >= J, of sum_{k in split c} Y[i][k] Y[j][k],
// stored transposed (entry (i, j) at [j][i], like the tensor-core partials);
// diagonal-tile CTAs also form sum_k Y[i][k] v[k].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_gram_simt(const T* __restrict__ A, long long lda, long long N, long long K,
            const int* __restrict__ idx, int sb, const double* __restrict__ v,
            long long chunks_per_split, int sbp, double* __restrict__ part,
            double* __restrict__ ppart, unsigned* __restrict__ err) {
  __shared__ double sA[64][33];
  __shared__ double sB[64][33];
  __shared__ double sv[32];
  __shared__ long long offA[64], offB[64];
  const int c = blockIdx.x;
  int tI, tJ;
  tri_decode(blockIdx.y, tI, tJ);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long k_begin = (long long)c * chunks_per_split * 32;
  const long long k_end = min(K, k_begin + chunks_per_split * 32);
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0.0;
  double pacc = 0.0;
  const bool diag = (tI == tJ);
  if (tid < 128) {  // row offsets, bounds-checked once (out of range: flagged, read as zero)
    const int r = tid & 63;
    const int gr = (tid < 64 ? tI : tJ) * 64 + r;
    long long off = -1;
    if (gr < sb) {
      const long long gi = idx[gr];
      if (gi >= 0 && gi < N) off = gi * lda;
      else ca_flag(err, CA_DEV_ERR_ARG);
    }
    (tid < 64 ? offA : offB)[r] = off;
  }
  __syncthreads();
  for (long long k0 = k_begin; k0 < k_end; k0 += 32) {
    for (int e = tid; e < 64 * 32; e += 256) {
      const int r = e >> 5, kk = e & 31;
      const long long k = k0 + kk;
      sA[r][kk] = (offA[r] >= 0 && k < k_end) ? (double)A[offA[r] + k] : 0.0;
      sB[r][kk] = (offB[r] >= 0 && k < k_end) ? (double)A[offB[r] + k] : 0.0;
    }
    if (tid < 32) sv[tid] = (k0 + tid < k_end) ? v[k0 + tid] : 0.0;
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      double a[4], bq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = sA[ty * 4 + q][kk];
        bq[q] = sB[tx * 4 + q][kk];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], bq[q], acc[p][q]);
    }
    if (diag && tid < 64) {
      for (int kk = 0; kk < 32; ++kk) pacc = fma(sA[tid][kk], sv[kk], pacc);
    }
    __syncthreads();
  }
  double* P = part + (long long)c * sbp * sbp;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      P[(long long)(tJ * 64 + tx * 4 + q) * sbp + (tI * 64 + ty * 4 + p)] = acc[p][q];
  if (diag && tid < 64) ppart[(long long)c * sbp + tI * 64 + tid] = pacc;
}

template __global__ void k_gram_simt<double>(const double*, long long, long long, long long,
                                             const int*, int, const double*, long long, int,
                                             double*, double*, unsigned*);
template __global__ void k_gram_simt<float>(const float*, long long, long long, long long,
                                            const int*, int, const double*, long long, int, double*,
                                            double*, unsigned*);

// ---------------------------------------------------------------------------
// a4: the s unrolled b x b solves of one outer step (eq. "recur" and its dual
// analogue), one CTA, FP64, in the block forward-substitution form
//   (cG R_jj + cI I) Delta_j = cP p_j - cI x[I_j] - cY yv[I_j] - cG sum_{t<j} R_jt Delta_t
// with x updated in place after each block, so that reading x[I_j] includes
// the index-overlap terms lambda I_j^T I_t Delta_t (primal) and
// I_j^T I_t Delta alpha_t (dual).  Shared memory: acc[sb], L[b*b], sol[b].
// ---------------------------------------------------------------------------
__device__ void block_solve(const double* __restrict__ R, const double* __restrict__ pvec,
                            const SolveArgs& a, unsigned* err, double* smem) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int b = a.b, sb = a.sb, ldr = a.ldr;
  double* acc = smem;            // sb
  double* L = acc + sb;          // b*b
  double* sol = L + (size_t)b * b;  // b
  for (int r = tid; r < sb; r += nt) acc[r] = a.cP * pvec[r];
  __syncthreads();
  for (int j = 0; j < a.s_cur; ++j) {
    const int base = j * b;
    // Gamma_j = cG R_jj + cI I (lower triangle) and the right-hand side
    for (int e = tid; e < b * b; e += nt) {
      const int p = e / b, q = e % b;
      if (q <= p)
        L[e] = a.cG * R[(long long)(base + p) * ldr + (base + q)] + (p == q ? a.cI : 0.0);
    }
    for (int p = tid; p < b; p += nt) {
      const int gi = a.idx[base + p];
      double r = acc[base + p];
      if (gi >= 0 && gi < a.N) {
        r -= a.cI * a.x[gi];
        if (a.yv) r -= a.cY * a.yv[gi];
      } else {
        ca_flag(err, CA_DEV_ERR_ARG);
      }
      sol[p] = r;
    }
    __syncthreads();
    // Cholesky Gamma_j = L L^T, right-looking, in place
    for (int col = 0; col < b; ++col) {
      if (tid == 0) {
        const double dgn = L[col * b + col];
        if (!(dgn > 0.0)) {
          ca_flag(err, isfinite(dgn) ? CA_DEV_ERR_NOT_SPD : CA_DEV_ERR_NONFINITE);
          L[col * b + col] = 1.0;
        } else {
          L[col * b + col] = sqrt(dgn);
        }
      }
      __syncthreads();
      const double piv = L[col * b + col];
      for (int r = col + 1 + tid; r < b; r += nt) L[r * b + col] /= piv;
      __syncthreads();
      const int rem = b - col - 1;
      for (int e = tid; e < rem * rem; e += nt) {
        const int r = col + 1 + e / rem, c2 = col + 1 + e % rem;
        if (c2 <= r) L[r * b + c2] -= L[r * b + col] * L[c2 * b + col];
      }
      __syncthreads();
    }
    // L u = rhs, L^T Delta = u  (warp 0; lanes split each dot product)
    if (tid < 32) {
      for (int i = 0; i < b; ++i) {
        double s = 0.0;
        for (int k = tid; k < i; k += 32) s += L[i * b + k] * sol[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (tid == 0) sol[i] = (sol[i] - s) / L[i * b + i];
        __syncwarp();
      }
      for (int i = b - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + tid; k < b; k += 32) s += L[k * b + i] * sol[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (tid == 0) sol[i] = (sol[i] - s) / L[i * b + i];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int p = tid; p < b; p += nt) {
      const double dl = sol[p];
      if (!isfinite(dl)) ca_flag(err, CA_DEV_ERR_NONFINITE);
      a.delta[base + p] = dl;
      const int gi = a.idx[base + p];
      if (gi >= 0 && gi < a.N) a.x[gi] += dl;  // no repeats inside a block
    }
    // right-looking update of the later blocks' right-hand sides
    for (int r = base + b + tid; r < sb; r += nt) {
      double s = 0.0;
      const double* Rr = R + (long long)r * ldr + base;
      for (int q = 0; q < b; ++q) s += Rr[q] * sol[q];
      acc[r] -= a.cG * s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// a4, fast form (b <= 32, s*b <= 256).  The diagonal blocks
// Gamma_j = cG R_jj + cI I are independent of the iterates, so they are
// factored and inverted up front (one CTA per block, in parallel); the
// dependent chain over j then needs no division or square root:
//   rhs_j   = cP p_j - cI x0[I_j] - cY y[I_j]
//             - sum_{t<j} (cG R_jt + cI [I_j == I_t]) Delta_t
//   Delta_j = Gamma_j^{-1} rhs_j
// where x0 is x at the start of the outer step; the index-equality term is the
// lambda I_j^T I_t Delta_t (primal) / I_j^T I_t Delta alpha_t (dual) overlap
// term of eq. "recur" and its dual analogue.  x is updated once per block at
// the end (atomic adds: an index may recur across blocks).
// ---------------------------------------------------------------------------

// Reduce the split-K partials (entry (i, j), i >= j, of partial c at
// part[c][j][i]) into R (lower triangle) and p.  Rs (when not
// null) receives the cG-scaled FP32 pairs of the lower-triangle entries,
// stored transposed (entry (i, j), i >= j, at Rs[j * ldr + i]) so that the
// chain reads a column block with coalesced loads.  CTAs 0 .. ndiag-1 each
// reduce one diagonal block Gamma_j = cG R_jj + cI I (b <= 16) and invert it
// into Ginv[j] (cta_sweep_inverse; two warps for b <= 8); the other CTAs take
// 64 entries per pass (warps 0-3: the first 32, one per lane; warps 4-7: the
// next 32), the 4 warps of a group splitting the P partials, so that every
// load of a pass is in flight at once.  Sums are double-float; R is written
// in FP64.
template <typename PT>
__device__ void reduce_body(const PT* __restrict__ part, const double* __restrict__ ppart, int P,
                            int sbp, double* __restrict__ R, float2* __restrict__ Rs,
                            double* __restrict__ pvec, float2* __restrict__ Ginv, int ndiag,
                            const SolveArgs& sa, unsigned* __restrict__ err, int cta, int ncta) {
  __shared__ float2 red[8][32];
  __shared__ float2 Mb[256];
  __shared__ float2 colbuf[66];
  __shared__ double redp[8][32];
  const int sb = sa.sb, ldr = sa.ldr;
  const long long sq = (long long)sbp * sbp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float2 cG2 = split_f64(sa.cG), cI2 = split_f64(sa.cI);
  if (cta < ndiag && sa.b <= 8) {
    // thread t sums row i = t % 8 of column jc = (t / 8) % 8 of the block
    // over the partials c = t / 64 (mod 4): a warp's load covers 4 columns x
    // 8 rows of one partial, four 32-byte sectors (entry (i, jc) of partial
    // c at part[c][base + jc][base + i])
    const int b = sa.b, base = cta * b;
    const int i = tid & 7, jc = (tid >> 3) & 7, sl = tid >> 6;
    float2* flat = &red[0][0];  // [4][64]
    flat[tid] = (i < b && jc < b && i >= jc)
                    ? sum_partials<PT, 40>(part + (long long)(base + jc) * sbp + (base + i), sl, P, 4, sq)
                    : make_float2(0.f, 0.f);
    __syncthreads();
    if (tid < 64 && i < b && jc < b && i >= jc) {
      const float2 t = df_add(df_add(flat[tid], flat[64 + tid]), df_add(flat[128 + tid], flat[192 + tid]));
      float2 v = df_mul(cG2, t);
      if (i == jc) v = df_add(v, cI2);
      Mb[i * b + jc] = v;
      Mb[jc * b + i] = v;
    }
    __syncthreads();
    if (tid < 64) {
      float2 a[1] = {tid < b * b ? Mb[tid] : make_float2(0.f, 0.f)};
      cta_sweep_inverse<1, 64>(a, b, colbuf, Ginv + (long long)cta * b * b, err);
    }
    return;
  }
  if (cta < ndiag) {
    const int b = sa.b, base = cta * b;
    const int E = b * (b + 1) / 2;
    const int nsl = 256 / E;  // >= 1 for b <= 16
    const int sl = tid / E, e = tid - sl * E;
    float2* flat = &red[0][0];
    if (sl < nsl) {
      int i, j;
      tri_decode(e, i, j);
      flat[tid] = sum_partials(part + (long long)(base + j) * sbp + (base + i), sl, P, nsl, sq);
    }
    __syncthreads();
    if (tid < E) {
      float2 t = make_float2(0.f, 0.f);
      for (int q = 0; q < nsl; ++q) t = df_add(t, flat[q * E + tid]);
      int i, j;
      tri_decode(tid, i, j);
      float2 v = df_mul(cG2, t);
      if (i == j) v = df_add(v, cI2);
      Mb[i * b + j] = v;
      Mb[j * b + i] = v;
    }
    __syncthreads();
    float2 a[1] = {tid < b * b ? Mb[tid] : make_float2(0.f, 0.f)};
    cta_sweep_inverse<1>(a, b, colbuf, Ginv + (long long)cta * b * b, err);
    return;
  }
  const long long nlow = (long long)sb * (sb + 1) / 2;
  const long long stride = (long long)(ncta - ndiag) * 64;
  const int grp = warp >> 2, sub = warp & 3;
  for (long long e0 = (long long)(cta - ndiag) * 64; e0 < nlow + sb; e0 += stride) {
    const long long e = e0 + grp * 32 + lane;
    int i = 0, j = 0;
    int kind = 0;  // 0 none, 1 Gram entry, 2 projection entry
    float2 s2 = make_float2(0.f, 0.f);
    double sp = 0.0;
    if (e < nlow) {
      // column-major over the lower triangle (consecutive lanes: consecutive
      // i of one column j), matching the transposed partials [j][i]
      int ir, jr;
      tri_decode(e, ir, jr);
      i = sb - 1 - jr;
      j = sb - 1 - ir;
      kind = 1;
    } else if (e < nlow + sb) {
      kind = 2;
      i = (int)(e - nlow);
    }
    if (kind == 1) {
      s2 = sum_partials<PT, 40>(part + (long long)j * sbp + i, sub, P, 4, sq);
    } else if (kind == 2) {
      const float2 q = sum_partials<double, 40>(ppart + i, sub, P, 4, (long long)sbp);
      sp = (double)q.x + (double)q.y;
    }
    red[warp][lane] = s2;
    redp[warp][lane] = sp;
    __syncthreads();
    if (sub == 0 && kind) {  // warps 0 and 4: the group's four sums
      const int w = warp;
      if (kind == 1) {
        const float2 t = df_add(df_add(red[w][lane], red[w + 1][lane]),
                                df_add(red[w + 2][lane], red[w + 3][lane]));
        R[(long long)i * ldr + j] = (double)t.x + (double)t.y;
        if (Rs) Rs[(long long)j * ldr + i] = df_mul(cG2, t);
      } else {
        pvec[i] = (redp[w][lane] + redp[w + 1][lane]) + (redp[w + 2][lane] + redp[w + 3][lane]);
      }
    }
    __syncthreads();
  }
}

template <typename PT>
__global__ void __launch_bounds__(256)
k_reduce(const PT* __restrict__ part, const double* __restrict__ ppart, int P, int sbp,
         double* __restrict__ R, float2* __restrict__ Rs, double* __restrict__ pvec,
         float2* __restrict__ Ginv, int ndiag, SolveArgs sa, unsigned* __restrict__ err) {
  reduce_body<PT>(part, ppart, P, sbp, R, Rs, pvec, Ginv, ndiag, sa, err, (int)blockIdx.x,
                  (int)gridDim.x);
}

template __global__ void k_reduce<double>(const double*, const double*, int, int, double*, float2*,
                                          double*, float2*, int, SolveArgs, unsigned*);
template __global__ void k_reduce<float>(const float*, const double*, int, int, double*, float2*,
                                         double*, float2*, int, SolveArgs, unsigned*);

// Gamma_j^{-1} for every diagonal block j = blockIdx.x from R (FP64 lower
// triangle), one CTA each (b <= 32).
__global__ void __launch_bounds__(256)
k_factor(const double* __restrict__ R, SolveArgs sa, float2* __restrict__ Ginv,
         unsigned* __restrict__ err) {
  __shared__ float2 colbuf[66];
  const int b = sa.b, base = (int)blockIdx.x * b;
  float2 a[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = (int)threadIdx.x + 256 * q;
    a[q] = make_float2(0.f, 0.f);
    if (e < b * b) {
      const int i = e / b, c = e - (e / b) * b;
      const int hi = i > c ? i : c, lo = i > c ? c : i;
      a[q] = split_f64(sa.cG * R[(long long)(base + hi) * sa.ldr + (base + lo)] + (i == c ? sa.cI : 0.0));
    }
  }
  cta_sweep_inverse<4>(a, b, colbuf, Ginv + (long long)blockIdx.x * b * b, err);
}

// The dependent chain (one CTA of 256 threads), for sb <= 256, b <= BMAX <= 32,
// with the diagonal-block inverses Ginv already formed.  Right-looking:
// thread r owns row r and keeps the sum
// acc_r = sum_{t solved} (cG R_rt + cI [I_r = I_t]) Delta_t; after block j is
// solved every later row folds in its b new terms, and the rows of block j+1
// then hold their complete right-hand sides.  The entries cG R[r][jb + q]
// arrive as FP32 pairs from the transposed Rs (column jb + q contiguous over
// r): the CTA streams the b columns of step j, DEPTH steps ahead, through a
// shared-memory ring with 16-byte cp.async.cg copies of row pairs (slot
// layout [q][row]: coalesced copies, conflict-free reads).  Everything the
// chain reads that an earlier kernel, or other CTAs of the same kernel, wrote
// is read through L2 (.cg / __ldcg), never from a possibly stale L1 line.
// Products are summed as trees (short dependency chains); everything on the
// dependent path is double-float; FP64 converts in at the start and out at
// the end.  256 threads; smem_d: the chain's dynamic shared memory.
template <int BMAX, int DEPTH>
__device__ void chain_body(const float2* __restrict__ Rs, const double* __restrict__ pvec,
                           const float2* __restrict__ Ginv, const SolveArgs& a,
                           unsigned* __restrict__ err, double* smem_d) {
  const int r = threadIdx.x;
  const int b = a.b, sb = a.sb, ldr = a.ldr, s = a.s_cur;
  float2* ring = reinterpret_cast<float2*>(smem_d);        // DEPTH x BMAX x 256
  float2* Gs = ring + (size_t)DEPTH * 256 * BMAX;          // sb*b: Gamma_j^{-1}
  float2* rb = Gs + (size_t)sb * b;                         // 32: rhs of the current block
  float2* dl = rb + 32;                                     // 32: Delta of the current block
  float2* dall = dl + 32;                                   // sb: all Delta
  int* sidx = reinterpret_cast<int*>(dall + sb);            // sb
  const uint32_t ring0 = smem_u32(ring);
  // 16-byte copies of row pairs need an even leading dimension (callers use
  // multiples of 32); otherwise nothing is copied and the call is flagged
  const bool ld_ok = (ldr & 1) == 0;
  if (!ld_ok && r == 0) ca_flag(err, CA_DEV_ERR_ARG);
  auto fetch = [&](int j) {  // columns jb .. jb+b of rows >= jb + b into slot j % DEPTH
    const int jb = j * b;
    if (j < s && ld_ok) {
      const int p0 = (jb + b) >> 1, np = ((sb + 1) >> 1) - p0;  // row pairs 2p, 2p+1
      for (int u = r; u < b * np; u += 256) {
        const int q = u / np, pr = 2 * (p0 + u - q * np);
        cp_async_16_zfill(ring0 + 8u * (uint32_t)(((j % DEPTH) * BMAX + q) * 256 + pr),
                          Rs + (long long)(jb + q) * ldr + pr, 16u);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int d = 0; d < DEPTH; ++d) fetch(d);
  for (int e = r; e < sb * b; e += 256) Gs[e] = __ldcg(Ginv + e);
  float2 rhs0 = make_float2(0.f, 0.f);
  int gi = -1;
  if (r < sb) {
    gi = a.idx[r];
    double v = a.cP * __ldcg(pvec + r);
    if (gi >= 0 && gi < a.N) {
      v -= a.cI * __ldcg(a.x + gi);
      if (a.yv) v -= a.cY * a.yv[gi];
    } else {
      ca_flag(err, CA_DEV_ERR_ARG);
    }
    rhs0 = split_f64(v);
    sidx[r] = gi;
    if (r < b) rb[r] = rhs0;  // block 0 has no earlier blocks
  }
  const float2 cI2 = split_f64(a.cI);
  float2 acc = make_float2(0.f, 0.f);    // row r: sum over the solved blocks
  float2 ovl = make_float2(0.f, 0.f);    // index-overlap sum of row r (rare)
  // Gamma_j^{-1} rhs_j: L lanes per row, each a strided share of the b terms
  constexpr int L = BMAX <= 16 ? BMAX : 8;
  const int grow = r / L, glane = r & (L - 1);
  __syncthreads();
  for (int j = 0; j < s; ++j) {
    const int jb = j * b;
    {  // every lane takes part in the shuffles (rows >= b contribute zero)
      float2 t = make_float2(0.f, 0.f);
      if (grow < b) {
        const float2* gr = Gs + (size_t)j * b * b + grow * b;
        for (int q = glane; q < b; q += L) t = df_add(t, df_mul(gr[q], rb[q]));
      }
#pragma unroll
      for (int o = L / 2; o >= 1; o /= 2) {
        const float2 u = make_float2(__shfl_xor_sync(0xffffffffu, t.x, o, L),
                                     __shfl_xor_sync(0xffffffffu, t.y, o, L));
        t = df_add(t, u);
      }
      if (grow < b && glane == 0) {
        dl[grow] = t;
        dall[jb + grow] = t;
      }
    }
    cp_async_wait<DEPTH - 1>();  // this thread's copies for step j have landed
    __syncthreads();             // ... and everyone else's
    if (r >= jb + b && r < sb) {  // fold block j into the later rows
      const float2* sl = ring + (size_t)(j % DEPTH) * BMAX * 256 + r;
      float2 pr[BMAX];
#pragma unroll
      for (int q = 0; q < BMAX; ++q) {
        pr[q] = make_float2(0.f, 0.f);
        if (q < b) {
          const float2 dq = dl[q];
          pr[q] = df_mul(sl[q * 256], dq);
          if (sidx[jb + q] == gi) ovl = df_add(ovl, dq);
        }
      }
      acc = df_add(acc, df_tree_sum(pr));
      if (r < jb + 2 * b) rb[r - jb - b] = df_add(rhs0, df_neg(df_add(acc, df_mul(cI2, ovl))));
    }
    __syncthreads();  // slot j % DEPTH is free only once every thread has folded
    fetch(j + DEPTH);
  }
  cp_async_wait<0>();
  if (r < sb) {  // Delta out, x += Delta (atomic: an index may recur across blocks)
    const float2 d2 = dall[r];
    const double dv = (double)d2.x + (double)d2.y;
    if (!isfinite(dv)) ca_flag(err, CA_DEV_ERR_NONFINITE);
    a.delta[r] = dv;
    if (gi >= 0 && gi < a.N) atomicAdd(a.x + gi, dv);
  }
}

template <int BMAX, int DEPTH>
__global__ void __launch_bounds__(256)
k_chain(const float2* __restrict__ Rs, const double* __restrict__ pvec,
        const float2* __restrict__ Ginv, SolveArgs a, unsigned* __restrict__ err) {
  extern __shared__ double smem_d[];
  pdl_wait();  // (as a programmatic dependent: p from the launch before it)
  if constexpr (BMAX <= 16)
    chain_la_body<BMAX, DEPTH>(Rs, pvec, Ginv, a, err, smem_d);
  else
    chain_body<BMAX, DEPTH>(Rs, pvec, Ginv, a, err, smem_d);
}

// a4 in one launch (b <= 16): CTAs 0 .. G-2 reduce (reduce_body, with the
// diagonal-block inverses) and count themselves done on *ticket; the last CTA
// runs the chain: it gathers what does not depend on the reduction (sampled
// indices, x0 and y there) while the others reduce, then waits (bounded) for
// the count.  Every CTA of the grid is resident before the next grid in the
// stream can start, and none of them waits for anything but this grid's
// reducing CTAs.  Launched as a programmatic dependent of the Gram pass: it
// waits for that grid, then lets the next Gram pass launch its CTAs, which
// prepare and start their loads on the SMs this grid frees while the chain
// runs.  *ticket is zero on entry and left zero.
template <typename PT, int BMAX, int DEPTH>
__global__ void __launch_bounds__(256)
k_reduce_chain(const PT* __restrict__ part, const double* __restrict__ ppart, int P, int sbp,
               double* __restrict__ R, float2* __restrict__ Rs, double* __restrict__ pvec,
               float2* __restrict__ Ginv, int ndiag, SolveArgs sa, unsigned* __restrict__ err,
               unsigned* __restrict__ ticket) {
  extern __shared__ double smem_d[];
  pdl_wait();
  pdl_trigger();
  const int nred = (int)gridDim.x - 1;
  if ((int)blockIdx.x < nred) {
    reduce_body<PT>(part, ppart, P, sbp, R, Rs, pvec, Ginv, ndiag, sa, err, (int)blockIdx.x, nred);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this CTA's R, Rs, p, Ginv before its count
      atomicAdd(ticket, 1u);
    }
    return;
  }
  chain_la_body<BMAX, DEPTH>(Rs, pvec, Ginv, sa, err, smem_d, ticket, (unsigned)nred);
}

template __global__ void k_reduce_chain<float, 8, 4>(const float*, const double*, int, int, double*,
                                                     float2*, double*, float2*, int, SolveArgs,
                                                     unsigned*, unsigned*);
template __global__ void k_reduce_chain<float, 16, 3>(const float*, const double*, int, int,
                                                      double*, float2*, double*, float2*, int,
                                                      SolveArgs, unsigned*, unsigned*);
template __global__ void k_reduce_chain<double, 8, 4>(const double*, const double*, int, int,
                                                      double*, float2*, double*, float2*, int,
                                                      SolveArgs, unsigned*, unsigned*);
template __global__ void k_reduce_chain<double, 16, 3>(const double*, const double*, int, int,
                                                       double*, float2*, double*, float2*, int,
                                                       SolveArgs, unsigned*, unsigned*);

// Shared launches over several problems (the batched solves): one grid
// reduces every problem's split-K partials (role table: problem and CTA index
// within it), one grid runs one chain CTA per problem.  No CTA waits on
// another, so neither grid needs its CTAs resident at once.
__global__ void __launch_bounds__(256)
k_reduce_batch(const RedInst* __restrict__ insts, const RedRole* __restrict__ roles,
               unsigned* __restrict__ err) {
  pdl_wait();
  pdl_trigger();
  const RedRole ro = roles[blockIdx.x];
  const RedInst ri = insts[ro.inst];
  reduce_body<float>(ri.part, ri.ppart, ri.P, ri.sbp, ri.R, ri.Rs, ri.pvec, ri.Ginv, ri.ndiag,
                     ri.sa, err, ro.cta, ro.ncta);
}

template <int BMAX, int DEPTH>
__global__ void __launch_bounds__(256)
k_chain_batch(const RedInst* __restrict__ insts, unsigned* __restrict__ err) {
  extern __shared__ double smem_d[];
  pdl_wait();
  pdl_trigger();
  const RedInst ri = insts[blockIdx.x];
  chain_la_body<BMAX, DEPTH>(ri.Rs, ri.pvec, ri.Ginv, ri.sa, err, smem_d);
}

template __global__ void k_chain<8, 4>(const float2*, const double*, const float2*, SolveArgs,
                                       unsigned*);
template __global__ void k_chain<16, 3>(const float2*, const double*, const float2*, SolveArgs,
                                        unsigned*);
template __global__ void k_chain<32, 2>(const float2*, const double*, const float2*, SolveArgs,
                                        unsigned*);

// The solves alone (sparse path: R and p are formed directly).
__global__ void __launch_bounds__(256)
k_solve(const double* __restrict__ R, const double* __restrict__ pvec, SolveArgs sa,
        unsigned* __restrict__ err) {
  extern __shared__ double smem_d[];
  block_solve(R, pvec, sa, err, smem_d);
}

// ---------------------------------------------------------------------------
// a5: deferred update  v[k] -= cU * sum_r Y[r][k] Delta_r  (primal: rho -= Y^T
// Delta, i.e. z += Y^T Delta; dual: w -= Y Delta alpha/(lambda n)).
// FP64 X: FP64 FMAs.  FP32 X: Delta split into two FP32 halves, FP32 products
// and sums over the rows (compensated across the row groups), the update
// applied in double-float to the FP32-pair copy of v.  (The stopping test
// rebuilds v with exact products before each check, so these FP32 roundings
// never reach its gap or f(w).)
// ---------------------------------------------------------------------------
// CTA = 4 row groups x 64 threads; thread t of group g handles the 4
// consecutive k at (64 blockIdx + t) * 4 and the rows r = g (mod 4); group 0
// adds the groups' partial sums and writes v (and its FP32 split v2).
// PANEL (FP32 only): A stored as 32-column panels [K/32][N][32] (zero-padded).
template <typename T, bool PANEL>
__global__ void __launch_bounds__(256)
k_update_dense(const T* __restrict__ A, long long lda, long long N, long long K,
               const int* __restrict__ idx, int sb, const double* __restrict__ delta, double cU,
               double* __restrict__ v, float2* __restrict__ v2, unsigned* __restrict__ err) {
  using Acc = typename std::conditional<sizeof(T) == 8, double, float>::type;
  extern __shared__ unsigned char smem_u[];
  __shared__ Acc red[3][64][4];
  int* sidx = reinterpret_cast<int*>(smem_u);
  double* sdl = reinterpret_cast<double*>(smem_u + ((sb * 4 + 255) & ~255));
  float2* sdl2 = reinterpret_cast<float2*>(sdl);  // FP32 path: Delta as (hi, lo)
  for (int r = threadIdx.x; r < sb; r += blockDim.x) {
    int gi = idx[r];
    double dl = delta[r];
    if (gi < 0 || (long long)gi >= N) {  // flagged; the row is skipped
      if (blockIdx.x == 0) ca_flag(err, CA_DEV_ERR_ARG);
      gi = 0;
      dl = 0.0;
    }
    sidx[r] = gi;
    if constexpr (sizeof(T) == 8) sdl[r] = dl;
    else sdl2[r] = split_f64(dl);
  }
  __syncthreads();
  const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
  const long long k = ((long long)blockIdx.x * 64 + t) * 4;
  const int nk = k < K ? (int)min(4ll, K - k) : 0;
  Acc acc[4] = {0, 0, 0, 0};
  if (nk > 0) {
    if constexpr (sizeof(T) == 8) {
      for (int r = grp; r < sb; r += 4) {
        const T* row = A + (long long)sidx[r] * lda + k;
        const double dl = sdl[r];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (e < nk) acc[e] = fma((double)row[e], dl, acc[e]);
      }
    } else {
      const bool vec = PANEL || ((nk == 4) && ((lda & 3) == 0) &&
                                 ((reinterpret_cast<uintptr_t>(A) & 15) == 0));
      const long long pbase = (k >> 5) * N * 32 + (k & 31);
#pragma unroll 8
      for (int r = grp; r < sb; r += 4) {
        const float* row = reinterpret_cast<const float*>(A) +
                           (PANEL ? pbase + (long long)sidx[r] * 32 : (long long)sidx[r] * lda + k);
        const float2 d2 = sdl2[r];
        float x[4];
        if (vec) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(row));
          x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) x[e] = (e < nk) ? row[e] : 0.f;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] = fmaf(x[e], d2.x, fmaf(x[e], d2.y, acc[e]));
      }
    }
  }
  if (grp > 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) red[grp - 1][t][e] = acc[e];
  }
  __syncthreads();
  if (grp == 0 && nk > 0) {
    if constexpr (sizeof(T) == 8) {
      for (int e = 0; e < nk; ++e) {
        const double nv = v[k + e] - cU * (acc[e] + red[0][t][e] + red[1][t][e] + red[2][t][e]);
        v[k + e] = nv;
        if (v2) v2[k + e] = split_f64(nv);
      }
    } else {
      // FP32 X: the FP32-pair copy v2 is the state the tensor-core passes
      // keep current; update it in double-float and refresh v from it
      const float2 cU2 = split_f64(cU);
      for (int e = 0; e < nk; ++e) {
        float hi = acc[e], lo = 0.f;
        comp_add(hi, lo, red[0][t][e]);
        comp_add(hi, lo, red[1][t][e]);
        comp_add(hi, lo, red[2][t][e]);
        float th, tl;
        two_sum(hi, lo, th, tl);
        const float2 nv = df_add(v2[k + e], df_neg(df_mul(cU2, make_float2(th, tl))));
        v2[k + e] = nv;
        v[k + e] = (double)nv.x + (double)nv.y;
      }
    }
  }
}

template __global__ void k_update_dense<double, false>(const double*, long long, long long,
                                                       long long, const int*, int, const double*,
                                                       double, double*, float2*, unsigned*);
template __global__ void k_update_dense<float, false>(const float*, long long, long long, long long,
                                                      const int*, int, const double*, double,
                                                      double*, float2*, unsigned*);
template __global__ void k_update_dense<float, true>(const float*, long long, long long, long long,
                                                     const int*, int, const double*, double,
                                                     double*, float2*, unsigned*);

// ---------------------------------------------------------------------------
// a6: full recompute  v[k] = c0 * y0[k] + c1 * sum_{r < N} A[r][k] x[r]
// (primal: rho = y - X^T w, or z = X^T w; dual: w = -X alpha/(lambda n)).
// Grid (K-blocks, row splits); row splits add into v with FP64 atomics after
// split 0 wrote the c0 * y0 term.  FP32 A: x split in two FP32 halves,
// exact products summed in double-float over the split's rows, then FP64.
// PANEL (FP32 only): A stored as 32-column panels [K/32][N][32]
// (zero-padded).
// ---------------------------------------------------------------------------
template <typename T, bool PANEL>
__global__ void __launch_bounds__(256)
k_recompute_dense(const T* __restrict__ A, long long lda, long long N, long long K,
                  const double* __restrict__ x, const float2* __restrict__ x2, double c1,
                  long long rows_per_split, double* __restrict__ v,
                  const unsigned* __restrict__ nz) {
  // x = 0 (a solve started from zero): sum_r A[r] x[r] = 0, A is not read
  if (nz && *nz == 0u) return;
  const long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (k >= K) return;
  const int nk = (int)min(4ll, K - k);
  const long long r0 = (long long)blockIdx.y * rows_per_split;
  const long long r1 = min(N, r0 + rows_per_split);
  double acc[4] = {0, 0, 0, 0};
  if constexpr (sizeof(T) == 8) {
    for (long long r = r0; r < r1; ++r) {
      const double xr = x[r];
      const T* row = A + r * lda + k;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e < nk) acc[e] = fma((double)row[e], xr, acc[e]);
    }
  } else {
    // x split in FP32 halves (x2); exact products, double-float sums
    const bool vec = PANEL || ((nk == 4) && ((lda & 3) == 0) &&
                               ((reinterpret_cast<uintptr_t>(A) & 15) == 0));
    const long long pbase = (k >> 5) * N * 32 + (k & 31);
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (long long r = r0; r < r1; ++r) {
      const float2 xs = __ldg(x2 + r);
      const float* row = reinterpret_cast<const float*>(A) + (PANEL ? pbase + r * 32 : r * lda + k);
      float q[4];
      if (vec) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(row));
        q[0] = t.x; q[1] = t.y; q[2] = t.z; q[3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) q[e] = (e < nk) ? row[e] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) df_dot_acc(q[e], xs.x, xs.y, hi[e], lo[e]);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] = (double)hi[e] + (double)lo[e];
  }
  for (int e = 0; e < nk; ++e) atomicAdd(v + k + e, c1 * acc[e]);
}

template __global__ void k_recompute_dense<double, false>(const double*, long long, long long,
                                                          long long, const double*, const float2*,
                                                          double, long long, double*,
                                                          const unsigned*);
template __global__ void k_recompute_dense<float, true>(const float*, long long, long long, long long,
                                                        const double*, const float2*, double,
                                                        long long, double*, const unsigned*);
template __global__ void k_recompute_dense<float, false>(const float*, long long, long long, long long,
                                                  const double*, const float2*, double, long long,
                                                  double*, const unsigned*);

// v2[k] = (hi, lo) FP32 split of v[k]; zero for K <= k < Kpad
__global__ void k_split(const double* __restrict__ v, long long K, long long Kpad,
                        float2* __restrict__ v2) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < Kpad) v2[k] = k < K ? split_f64(v[k]) : make_float2(0.f, 0.f);
}

// v = c0 * y0 (or 0 when y0 is null); clears *nz (when not null) for k_nonzero
__global__ void k_axpby_init(const double* __restrict__ y0, double c0, long long K,
                             double* __restrict__ v, unsigned* __restrict__ nz) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) v[k] = y0 ? c0 * y0[k] : 0.0;
  if (nz && k == 0) *nz = 0u;
}

// *nz = 1 if any x[r] != 0 (r < N); x2 (when not null) receives the (hi, lo)
// FP32 split of x
__global__ void k_nonzero(const double* __restrict__ x, long long N, float2* __restrict__ x2,
                          unsigned* __restrict__ nz) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double xv = r < N ? x[r] : 0.0;
  if (x2 && r < N) x2[r] = split_f64(xv);
  if (__any_sync(0xffffffffu, xv != 0.0) && (threadIdx.x & 31) == 0) atomicOr(nz, 1u);
}

// ---------------------------------------------------------------------------
// Dual, sparse X (CSR of X^T, row i = column x_i of X, column indices sorted).
// ---------------------------------------------------------------------------
// Diagonal entries x_{I_p}^T x_{I_p} (exact products in FP64) and
// projections x_{I_p}^T w of the sampled rows, one warp per row.
__global__ void __launch_bounds__(256)
k_csr_rows(const long long* __restrict__ rowptr, const int* __restrict__ col,
           const float* __restrict__ val, const int* __restrict__ idx, long long nrows,
           long long ncols, int sb, int ldr, const double* __restrict__ w,
           double* __restrict__ G, double* __restrict__ pvec, unsigned* __restrict__ err) {
  pdl_wait();  // w (the previous step's update) and the previous use of G
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= sb) return;
  const int ir = idx[r];
  double sp = 0.0, sd = 0.0;
  if (ir >= 0 && ir < nrows) {
    const long long e1 = rowptr[ir + 1];
    for (long long eb = rowptr[ir] + lane; eb < e1; eb += 256) {
      // eight entries in flight per lane, then their gathers of w
      int fs[8];
      float vs[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const long long e = eb + 32 * u;
        fs[u] = e < e1 ? col[e] : -1;
        vs[u] = e < e1 ? val[e] : 0.f;
      }
      double ws[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool in = fs[u] >= 0 && fs[u] < ncols;
        if (!in && eb + 32 * u < e1) ca_flag(err, CA_DEV_ERR_ARG);
        ws[u] = in ? w[fs[u]] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        sd = fma((double)vs[u], (double)vs[u], sd);
        sp = fma((double)vs[u], ws[u], sp);
      }
    }
  } else if (lane == 0) {
    ca_flag(err, CA_DEV_ERR_ARG);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sp += __shfl_xor_sync(0xffffffffu, sp, o);
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
  }
  if (lane == 0) {
    pvec[r] = sp;
    G[(long long)r * ldr + r] = sd;
  }
}

// Projections x_{I_p}^T w of the sampled rows alone (the part of a2+a3 that
// needs the current w), one CTA per row: thread t takes entries t, t + 256,
// ... of the row, four in flight, then a CTA sum (FP64 products and sums).
__global__ void __launch_bounds__(256)
k_csr_proj(const long long* __restrict__ rowptr, const int* __restrict__ col,
           const float* __restrict__ val, const int* __restrict__ idx, long long nrows,
           long long ncols, const double* __restrict__ w, double* __restrict__ pvec,
           unsigned* __restrict__ err) {
  __shared__ double red[8];
  pdl_wait();  // w (the previous step's update)
  pdl_trigger();
  const int r = blockIdx.x, tid = threadIdx.x;
  const int ir = idx[r];
  double sp = 0.0;
  if (ir >= 0 && ir < nrows) {
    const long long e1 = rowptr[ir + 1];
    for (long long eb = rowptr[ir] + tid; eb < e1; eb += 4 * 256) {
      int fs[4];
      float vs[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long e = eb + 256 * u;
        fs[u] = e < e1 ? col[e] : -1;
        vs[u] = e < e1 ? val[e] : 0.f;
      }
      double ws[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = fs[u] >= 0 && fs[u] < ncols;
        if (!in && eb + 256 * u < e1) ca_flag(err, CA_DEV_ERR_ARG);
        ws[u] = in ? w[fs[u]] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) sp = fma((double)vs[u], ws[u], sp);
    }
  } else if (tid == 0) {
    ca_flag(err, CA_DEV_ERR_ARG);
  }
  for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
  if ((tid & 31) == 0) red[tid >> 5] = sp;
  __syncthreads();
  if (tid == 0)
    pvec[r] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
}

// rn[r] = x_r^T x_r for every row of the CSR (exact products, FP64 sums),
// one warp per row: the diagonal of every Gram, formed once per solve.
__global__ void __launch_bounds__(256)
k_csr_rownorm(const long long* __restrict__ rowptr, const float* __restrict__ val,
              long long nrows, double* __restrict__ rn) {
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nrows) return;
  const long long e1 = rowptr[r + 1];
  double sd = 0.0;
  for (long long eb = rowptr[r] + lane; eb < e1; eb += 8 * 32) {
    float vs[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) vs[u] = eb + 32 * u < e1 ? val[eb + 32 * u] : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) sd = fma((double)vs[u], (double)vs[u], sd);
  }
  for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
  if (lane == 0) rn[r] = sd;
}

// The part of a4's input that depends on neither w nor alpha (so it can be
// formed while the previous outer step still runs): CTAs 0 .. s'-1 take the
// diagonal block j: the diagonal from the row norms rn (k_csr_rownorm), the
// strict lower part from G, Gamma_j = cG G_jj + cI I in double-float and its
// inverse (cta_sweep_inverse) into Ginv[j];
// the other CTAs write Rs = cG G (FP32 pairs) over the strict lower
// triangle, in G's transposed layout (entry (i, c), i > c, at c * ldr + i),
// which is the layout the chain reads.  b <= 16.
__global__ void __launch_bounds__(256)
k_csr_prep(const double* __restrict__ rn, const int* __restrict__ idx, long long nrows,
           const double* __restrict__ G, SolveArgs sa, float2* __restrict__ Rs,
           float2* __restrict__ Ginv, unsigned* __restrict__ err) {
  __shared__ double dsum[16];
  __shared__ float2 Mb[256];
  __shared__ float2 colbuf[66];
  pdl_wait();  // G's strict lower triangle (the Gram kernels before this one)
  pdl_trigger();
  const int b = sa.b, sb = sa.sb, ldr = sa.ldr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float2 cG2 = split_f64(sa.cG), cI2 = split_f64(sa.cI);
  if ((int)blockIdx.x < sa.s_cur) {
    const int jb = (int)blockIdx.x * b;
    if (tid < b) {
      const int ir = idx[jb + tid];
      const bool ok = ir >= 0 && ir < nrows;
      if (!ok) ca_flag(err, CA_DEV_ERR_ARG);
      dsum[tid] = ok ? rn[ir] : 0.0;
    }
    __syncthreads();
    if (tid < b * b) {
      const int i = tid / b, c = tid - (tid / b) * b;
      const double v = i == c ? dsum[i]
                              : G[(long long)(jb + (i < c ? i : c)) * ldr + jb + (i < c ? c : i)];
      float2 m = df_mul(cG2, split_f64(v));
      if (i == c) m = df_add(m, cI2);
      Mb[tid] = m;
    }
    __syncthreads();
    float2* out = Ginv + (long long)blockIdx.x * b * b;
    if (b <= 8) {
      if (tid < 64) {
        float2 a[1] = {tid < b * b ? Mb[tid] : make_float2(0.f, 0.f)};
        cta_sweep_inverse<1, 64>(a, b, colbuf, out, err);
      }
    } else {
      float2 a[1] = {tid < b * b ? Mb[tid] : make_float2(0.f, 0.f)};
      cta_sweep_inverse<1>(a, b, colbuf, out, err);
    }
    return;
  }
  const long long ne = (long long)sb * sb;
  const long long stride = (long long)(gridDim.x - sa.s_cur) * 256;
  for (long long e = (long long)(blockIdx.x - sa.s_cur) * 256 + tid; e < ne; e += stride) {
    const int c = (int)(e / sb), i = (int)(e - (long long)c * sb);
    if (i > c) Rs[(long long)c * ldr + i] = df_mul(cG2, split_f64(G[(long long)c * ldr + i]));
  }
}

// The off-diagonal Gram entries of few sampled rows (s*b <= 64) by sorted-list
// intersection, one warp per pair q < p: lanes walk the shorter row and
// binary-search the longer, products exact in FP64.
__global__ void __launch_bounds__(256)
k_csr_gram_pairs(const long long* __restrict__ rowptr, const int* __restrict__ col,
                 const float* __restrict__ val, const int* __restrict__ idx, long long nrows,
                 int sb, int ldr, double* __restrict__ G) {
  pdl_wait();  // the previous use of G
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const long long npairs = (long long)sb * (sb - 1) / 2;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long e = warp; e < npairs; e += nwarps) {
    int p, q;
    tri_decode(e, p, q);  // q <= p over a triangle of side sb - 1
    p += 1;               // q < p
    const int ip = idx[p], iq = idx[q];
    double acc = 0.0;
    if (ip >= 0 && ip < nrows && iq >= 0 && iq < nrows) {
      long long a0 = rowptr[ip], a1 = rowptr[ip + 1];
      long long b0 = rowptr[iq], b1 = rowptr[iq + 1];
      if (a1 - a0 > b1 - b0) {
        long long t0 = a0, t1 = a1;
        a0 = b0; a1 = b1; b0 = t0; b1 = t1;
      }
      for (long long ea = a0 + lane; ea < a1; ea += 32) {
        const int f = col[ea];
        long long lo = b0, hi = b1;
        while (lo < hi) {
          const long long mid = (lo + hi) >> 1;
          if (col[mid] < f) lo = mid + 1; else hi = mid;
        }
        if (lo < b1 && col[lo] == f) acc = fma((double)val[ea], (double)val[lo], acc);
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) G[(long long)q * ldr + p] = acc;
  }
}

// The sparse Gram of one outer step (steps a2+a3, Alg. 4 "compute the Gram
// matrix" on the CSR of X^T): G[p][q] = x_{I_p}^T x_{I_q} for q < p.  The
// lower triangle is cut into tiles of kCsrPB
// rows p by kCsrQC rows q, one CTA each: the CTA puts its rows p into
// shared-memory hash tables (feature -> value), then its warps stream the
// rows q of the tile once, four entries per lane in flight, each entry
// probing every table.  The work is the streamed row lengths times the
// tables, with no atomics and each Gram entry written by one warp.  Products
// of two FP32 values are exact as (p, e) by a fused multiply-add and are
// summed in double-float (~2^-44 of sum |terms|); a row p longer than its
// table is searched in its sorted global columns instead.  The diagonal and
// the projections come from k_csr_rows.  The Gram goes out as the one split-K
// "partial" of the dense path's reduction (transposed: entry (i, j), i >= j,
// at G[j * ldr + i]).
constexpr int kCsrPB = 4;                      // rows p of a tile (rows q: qc, a launch argument)
constexpr int kCsrHashBits = 11;               // a table of 2048 entries per row p
constexpr int kCsrHash = 1 << kCsrHashBits;
constexpr int kCsrHashMaxRow = kCsrHash / 2;   // load factor <= 1/2
constexpr int kCsrSmem = kCsrPB * kCsrHash * 8;  // dynamic shared memory of k_csr_gram

__device__ __forceinline__ unsigned csr_hash(int f) {
  return ((unsigned)f * 2654435761u) >> (32 - kCsrHashBits);
}

// tiles of the lower triangle: row block pb has ceil(min(sb, (pb+1) PB) / qc)
__host__ __device__ __forceinline__ int csr_tiles_of(int pb, int sb, int qc) {
  const int pmax = min(sb, (pb + 1) * kCsrPB);
  return (pmax + qc - 1) / qc;
}

__global__ void __launch_bounds__(256)
k_csr_gram(const long long* __restrict__ rowptr, const int* __restrict__ col,
           const float* __restrict__ val, const int* __restrict__ idx, long long nrows,
           long long ncols, int sb, int ldr, int qcs, const double* __restrict__ w,
           double* __restrict__ G, double* __restrict__ pvec, unsigned* __restrict__ err) {
  // dynamic shared memory: kCsrPB tables of kCsrHash keys and values
  extern __shared__ int csr_smem[];
  int (*hkey)[kCsrHash] = reinterpret_cast<int (*)[kCsrHash]>(csr_smem);
  float (*hval)[kCsrHash] = reinterpret_cast<float (*)[kCsrHash]>(csr_smem + kCsrPB * kCsrHash);
  pdl_wait();  // w (the previous step's update) and the previous use of G
  pdl_trigger();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // this CTA's tile: row block pb, q chunk qc
  int pb = 0, rem = blockIdx.x;
  while (rem >= csr_tiles_of(pb, sb, qcs)) rem -= csr_tiles_of(pb, sb, qcs), ++pb;
  const int qc = rem;
  const int pl = pb * kCsrPB, ph = min(sb, pl + kCsrPB);  // rows p: [pl, ph)
  const int ql = qc * qcs, qh = min(ph, ql + qcs);         // rows q: [ql, qh), q <= p
  long long p0[kCsrPB], p1[kCsrPB];
  bool hashed[kCsrPB];
#pragma unroll
  for (int j = 0; j < kCsrPB; ++j) {
    const int p = pl + j;
    const int ip = p < ph ? idx[p] : -1;
    const bool okp = ip >= 0 && ip < nrows;
    if (p < ph && !okp && tid == 0) ca_flag(err, CA_DEV_ERR_ARG);
    p0[j] = okp ? rowptr[ip] : 0;
    p1[j] = okp ? rowptr[ip + 1] : 0;
    hashed[j] = p1[j] - p0[j] <= kCsrHashMaxRow;
  }
  for (int k = tid; k < kCsrPB * kCsrHash; k += 256) (&hkey[0][0])[k] = -1;
  __syncthreads();
  // the tables: every row p's entries, four loads in flight per thread
#pragma unroll
  for (int j = 0; j < kCsrPB; ++j) {
    if (!hashed[j]) continue;
    for (long long eb = p0[j] + tid; eb < p1[j]; eb += 1024) {
      int fs[4];
      float vs[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long e = eb + 256 * u;
        fs[u] = e < p1[j] ? col[e] : -1;
        vs[u] = e < p1[j] ? val[e] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (fs[u] < 0) continue;
        unsigned h = csr_hash(fs[u]);
        while (atomicCAS(&hkey[j][h], -1, fs[u]) != -1) h = (h + 1) & (kCsrHash - 1);
        hval[j][h] = vs[u];
      }
    }
  }
  __syncthreads();
  // value of feature f in row p = pl + j (0 when absent)
  auto lookup = [&](int j, int f) -> float {
    if (hashed[j]) {
      unsigned h = csr_hash(f);
      for (;;) {
        const int k = hkey[j][h];
        if (k == f) return hval[j][h];
        if (k == -1) return 0.f;
        h = (h + 1) & (kCsrHash - 1);
      }
    }
    long long lo = p0[j], hi = p1[j];  // a long row: its sorted global columns
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (col[mid] < f) lo = mid + 1; else hi = mid;
    }
    return (lo < p1[j] && col[lo] == f) ? val[lo] : 0.f;
  };
  for (int q = ql + warp; q < qh; q += 8) {
    const int iq = idx[q];
    float hi[kCsrPB], lo[kCsrPB];
#pragma unroll
    for (int j = 0; j < kCsrPB; ++j) hi[j] = lo[j] = 0.f;
    if (iq >= 0 && iq < nrows) {
      const long long e0 = rowptr[iq], e1 = rowptr[iq + 1];
      for (long long eb = e0 + lane; eb < e1; eb += 128) {
        int fs[4];
        float vs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // four entries in flight per lane
          const long long e = eb + 32 * u;
          fs[u] = e < e1 ? col[e] : -1;
          vs[u] = e < e1 ? val[e] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (fs[u] < 0) continue;
#pragma unroll
          for (int j = 0; j < kCsrPB; ++j) {
            if (pl + j <= q || pl + j >= ph) continue;  // pairs q < p (k_csr_rows: q = p)
            const float vp = lookup(j, fs[u]);
            if (vp != 0.f) {
              const float pr = vp * vs[u];
              const float pe = fmaf(vp, vs[u], -pr);  // vp vq = pr + pe exactly
              float s2, t2;
              two_sum(hi[j], pr, s2, t2);
              hi[j] = s2;
              lo[j] += t2 + pe;
            }
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kCsrPB; ++j) {
      if (pl + j <= q || pl + j >= ph) continue;
      float2 acc = df_norm(hi[j], lo[j]);
      for (int o = 16; o > 0; o >>= 1) acc = df_add(acc, df_shfl_xor(acc, o));
      if (lane == 0) G[(long long)q * ldr + pl + j] = (double)acc.x + (double)acc.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Sparse Gram by a dense-sparse split of the features (steps a2+a3 of Alg. 4
// on the CSR of X^T).  A feature present in a large share of the samples
// makes almost every sampled pair nonzero: its contribution to G = Y Y^T is
// a dense rank-one term, cheaper to form as part of a small dense Gram than
// pair by pair.  Once per solve the heavy features get a column of the dense
// n x fd matrix Xd (k_colcount, host choice, k_dense_fill); every outer step
// k_dgram forms the Gram of the sampled rows of Xd (exact products summed
// in double-float) and writes the strict lower triangle of G, then k_sgram
// adds the products of the remaining features: each CTA takes a range of
// features, gathers the sampled rows' entries in it (a binary search per row
// in its sorted columns), buckets them by feature in shared memory and adds
// the exact product of every pair of entries of a feature to G with FP64
// atomics.  Together with k_csr_rows (diagonal, projections) this is the
// same G as the pair kernels form, up to the order of FP64 additions.
// ---------------------------------------------------------------------------
// cnt[f] += 1 for every stored entry of column f (cnt zero on entry)
__global__ void __launch_bounds__(256)
k_colcount(const int* __restrict__ col, long long nnz, long long ncols, int* __restrict__ cnt) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x) {
    const int f = col[e];
    if (f >= 0 && f < ncols) atomicAdd(cnt + f, 1);
  }
}

// Xd[r][dmap[f]] = X^T[r][f] for the mapped (heavy) features (Xd zero on entry)
__global__ void __launch_bounds__(256)
k_dense_fill(const long long* __restrict__ rowptr, const int* __restrict__ col,
             const float* __restrict__ val, long long nrows, long long ncols,
             const int* __restrict__ dmap, int fd, float* __restrict__ Xd) {
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nrows) return;
  for (long long e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32) {
    const int f = col[e];
    const int j = (f >= 0 && f < ncols) ? dmap[f] : -1;
    if (j >= 0) Xd[r * fd + j] = val[e];
  }
}

constexpr int kDgT = 16;  // G tile of k_dgram: 16 x 16 entries, one per thread
constexpr int kCsrDenseMax = CA_CSR_DENSE_MAX;  // dense features at most

// G[q][p] (q < p, transposed: at G[q * ldr + p]) = x_{I_p}^T x_{I_q} over the
// dense features: exact products summed in double-float.  One CTA per 16 x 16
// tile of the lower triangle (tile pairs qb <= pb); fd = 0 writes zeros.  fd
// is a multiple of 8 (Xd's zero-padded row length, 16-byte rows).
__global__ void __launch_bounds__(256)
k_dgram(const float* __restrict__ Xd, int fd, const int* __restrict__ idx, int sb,
        long long nrows, int ldr, double* __restrict__ G) {
  extern __shared__ float4 dg_smem4[];  // [2 kDgT][(fd + 4) / 4]: rows p, then rows q
  float* dg_smem = reinterpret_cast<float*>(dg_smem4);
  pdl_wait();  // the previous use of G
  pdl_trigger();
  int pb, qb;
  tri_decode(blockIdx.x, pb, qb);
  // row stride fd + 4 floats: 16-byte rows whose 16-byte loads by 8
  // consecutive rows fall in distinct bank groups
  const int ld = fd + 4, n4 = fd >> 2;
  // the 2 kDgT rows into shared memory: every 16-byte copy in flight at once
  // (cp.async), rows outside the sample zero
  const uint32_t sm0 = smem_u32(dg_smem);
  for (int s = threadIdx.x >> 5; s < 2 * kDgT; s += 8) {  // a warp per row
    const int r = s < kDgT ? pb * kDgT + s : qb * kDgT + s - kDgT;
    const int i = r < sb ? idx[r] : -1;
    if (i >= 0 && i < nrows) {
      const float* src = Xd + (long long)i * fd;
      for (int f4 = threadIdx.x & 31; f4 < n4; f4 += 32)
        cp_async_16_zfill(sm0 + 4u * (uint32_t)(s * ld + 4 * f4), src + 4 * f4, 16u);
    } else {
      for (int f4 = threadIdx.x & 31; f4 < n4; f4 += 32)
        dg_smem4[(s * ld >> 2) + f4] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  const int ty = threadIdx.x / kDgT, tx = threadIdx.x % kDgT;
  const int p = pb * kDgT + ty, q = qb * kDgT + tx;
  if (p < sb && q < p) {
    const float4* yp = dg_smem4 + (ty * ld >> 2);
    const float4* yq = dg_smem4 + ((kDgT + tx) * ld >> 2);
    // four independent double-float sums (features f = u mod 4): four
    // dependency chains in flight instead of one; 16-byte loads
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int f4 = 0; f4 < n4; ++f4) {
      const float4 x = yp[f4], y = yq[f4];
      df_dot_acc(x.x, y.x, 0.f, hi[0], lo[0]);
      df_dot_acc(x.y, y.y, 0.f, hi[1], lo[1]);
      df_dot_acc(x.z, y.z, 0.f, hi[2], lo[2]);
      df_dot_acc(x.w, y.w, 0.f, hi[3], lo[3]);
    }
    const float2 s2 = df_add(df_add(df_norm(hi[0], lo[0]), df_norm(hi[1], lo[1])),
                             df_add(df_norm(hi[2], lo[2]), df_norm(hi[3], lo[3])));
    G[(long long)q * ldr + p] = (double)s2.x + (double)s2.y;
  }
}

constexpr int kSgFR = 512;    // features per CTA of k_sgram
constexpr int kSgCap = 4096;  // entries per pass (a range with more is split)
constexpr int kSgSmem = 3 * (kSgFR + 1) * 4 + kSgCap * (4 + 4 + 2) + kSgCap * (4 + 4) + 64;

// roff[r (nr + 1) + c] = the offset within row r of its first entry with
// column >= c kSgFR (the row's length when it has none), c = 0 .. nr: where
// each feature range of k_sgram starts in every row, formed once per solve
// so that k_sgram needs no search.  One warp per row.
__global__ void __launch_bounds__(256)
k_csr_rangeoff(const long long* __restrict__ rowptr, const int* __restrict__ col,
               long long nrows, int nr, int* __restrict__ roff) {
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nrows) return;
  const long long e0 = rowptr[r], e1 = rowptr[r + 1];
  int* out = roff + r * (nr + 1);
  auto range_of = [&](int f) { return f < 0 ? -1 : min(f / kSgFR, nr); };
  for (long long e = e0 + lane; e < e1; e += 32) {
    const int c = range_of(col[e]);
    const int cp = e == e0 ? -1 : range_of(col[e - 1]);
    for (int q = cp + 1; q <= c; ++q) out[q] = (int)(e - e0);
  }
  const int cl = e1 > e0 ? range_of(col[e1 - 1]) : -1;  // ranges after the last entry's
  for (int q = cl + 1 + lane; q <= nr; q += 32) out[q] = (int)(e1 - e0);
}

// G[q][p] (q < p) += products of the sampled rows' entries in the features
// dmap[f] < 0, FP64 atomics (G holds the dense part on entry).  roff (when
// not null, nr + 1 offsets a row, k_csr_rangeoff) gives where the CTA's
// range starts in each row; otherwise a binary search finds it.
__global__ void __launch_bounds__(256)
k_sgram(const long long* __restrict__ rowptr, const int* __restrict__ col,
        const float* __restrict__ val, const int* __restrict__ idx, long long nrows,
        long long ncols, int sb, const int* __restrict__ dmap, int ldr, double* __restrict__ G,
        const int* __restrict__ roff, int nr) {
  extern __shared__ int sg_smem[];
  int* cntf = sg_smem;                   // [kSgFR + 1] entries per feature
  int* off = cntf + (kSgFR + 1);         // [kSgFR + 1] their start (then a fill cursor)
  int* pc = off + (kSgFR + 1);           // [kSgFR + 1] pairs before feature f
  int* er = pc + (kSgFR + 1);            // [kSgCap] gathered: row slot
  float* ev = reinterpret_cast<float*>(er + kSgCap);       // value
  short* ef = reinterpret_cast<short*>(ev + kSgCap);       // feature within the range
  int* sr = reinterpret_cast<int*>(ef + kSgCap);           // bucketed: row slot
  float* sv = reinterpret_cast<float*>(sr + kSgCap);       // value
  int* scal = reinterpret_cast<int*>(sv + kSgCap);         // [0] entries gathered
  pdl_wait();  // G written by k_dgram
  pdl_trigger();
  const int tid = threadIdx.x;
  const long long f0 = (long long)blockIdx.x * kSgFR;
  const long long f1 = f0 + kSgFR < ncols ? f0 + kSgFR : ncols;
  long long fa = f0;
  while (fa < f1) {
    long long fb = f1;
    for (;;) {  // gather [fa, fb); halve the range while it holds too many entries
      for (int k = tid; k <= kSgFR; k += 256) cntf[k] = 0;
      if (tid == 0) scal[0] = 0;
      __syncthreads();
      for (int r = tid; r < sb; r += 256) {
        const int i = idx[r];
        if (i < 0 || i >= nrows) continue;
        long long lo = rowptr[i], hi = rowptr[i + 1];
        const long long end = hi;
        if (roff && fa == f0) {
          lo += roff[(long long)i * (nr + 1) + blockIdx.x];
        } else {
          while (lo < hi) {  // first entry with column >= fa
            const long long mid = (lo + hi) >> 1;
            if (col[mid] < fa) lo = mid + 1; else hi = mid;
          }
        }
        for (long long e = lo; e < end; ++e) {
          const int f = col[e];
          if (f >= fb) break;
          if (dmap[f] >= 0) continue;
          const int pos = atomicAdd(scal, 1);
          if (pos < kSgCap) {
            er[pos] = r;
            ev[pos] = val[e];
            ef[pos] = (short)(f - fa);
            atomicAdd(cntf + (f - fa), 1);
          }
        }
      }
      __syncthreads();
      if (scal[0] <= kSgCap || fb - fa <= 1) break;  // (one feature holds <= sb <= kSgCap)
      fb = fa + (fb - fa) / 2;
      __syncthreads();
    }
    const int ne = scal[0] < kSgCap ? scal[0] : kSgCap;
    const int nf = (int)(fb - fa);
    {  // offsets and pair counts: exclusive scans over the nf <= 512 features,
       // two per thread, then across the warps
      const int fa2 = 2 * tid, fb2 = 2 * tid + 1;
      const int c0 = fa2 < nf ? cntf[fa2] : 0, c1 = fb2 < nf ? cntf[fb2] : 0;
      int so = c0 + c1, sq = c0 * (c0 - 1) / 2 + c1 * (c1 - 1) / 2;
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {  // inclusive warp scans
        const int xo = __shfl_up_sync(0xffffffffu, so, o), xq = __shfl_up_sync(0xffffffffu, sq, o);
        if (lane >= o) {
          so += xo;
          sq += xq;
        }
      }
      __shared__ int wtot[2][8];
      if (lane == 31) {
        wtot[0][warp] = so;
        wtot[1][warp] = sq;
      }
      __syncthreads();
      int bo = 0, bq = 0;
      for (int w2 = 0; w2 < warp; ++w2) {
        bo += wtot[0][w2];
        bq += wtot[1][w2];
      }
      const int eo = bo + so - (c0 + c1), eq = bq + sq - (c0 * (c0 - 1) / 2 + c1 * (c1 - 1) / 2);
      if (fa2 < nf) {
        off[fa2] = eo;
        pc[fa2] = eq;
      }
      if (fb2 < nf) {
        off[fb2] = eo + c0;
        pc[fb2] = eq + c0 * (c0 - 1) / 2;
      }
      if (tid == 255) {
        off[nf] = bo + so;
        pc[nf] = bq + sq;
      }
    }
    __syncthreads();
    for (int e = tid; e < ne; e += 256) {  // bucket by feature
      const int f = ef[e];
      const int pos = off[f] + atomicAdd(cntf + f, -1) - 1;
      sr[pos] = er[e];
      sv[pos] = ev[e];
    }
    __syncthreads();
    const int np = pc[nf];
    for (int t = tid; t < np; t += 256) {
      int lo = 0, hi = nf;  // feature f: pc[f] <= t < pc[f + 1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pc[mid] <= t) lo = mid; else hi = mid;
      }
      int a, b2;
      tri_decode(t - pc[lo], a, b2);  // b2 <= a over side c - 1: the pair (b2, a + 1)
      const int base = off[lo];
      const int r1 = sr[base + b2], r2 = sr[base + a + 1];
      const int p = r1 > r2 ? r1 : r2, q = r1 > r2 ? r2 : r1;
      atomicAdd(G + (long long)q * ldr + p, (double)sv[base + b2] * (double)sv[base + a + 1]);
    }
    __syncthreads();
    fa = fb;
  }
}

// v[col] += c * val * coef[r] for the listed rows (a5 for CSR with coef =
// Delta alpha, c = -1/(lambda n); a6 with all rows, coef = alpha).
__global__ void __launch_bounds__(256)
k_scatter_csr(const long long* __restrict__ rowptr, const int* __restrict__ col,
              const float* __restrict__ val, const int* __restrict__ idx, long long nrows_total,
              long long ncols, long long nlist, const double* __restrict__ coef, double c,
              double* __restrict__ v, unsigned* __restrict__ err) {
  pdl_wait();  // (launched as a programmatic dependent of the solve)
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nlist) return;
  const long long row = idx ? (long long)idx[r] : r;
  if (row < 0 || row >= nrows_total) {
    if (lane == 0) ca_flag(err, CA_DEV_ERR_ARG);
    return;
  }
  const double cr = c * coef[r];
  const long long e1 = rowptr[row + 1];
  for (long long eb = rowptr[row] + lane; eb < e1; eb += 256) {
    int fs[8];  // eight entries in flight per lane
    float vs[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long e = eb + 32 * u;
      fs[u] = e < e1 ? col[e] : -1;
      vs[u] = e < e1 ? val[e] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (fs[u] >= 0 && fs[u] < ncols) atomicAdd(v + fs[u], (double)vs[u] * cr);
      else if (eb + 32 * u < e1) ca_flag(err, CA_DEV_ERR_ARG);
    }
  }
}

// a5 for the sampled rows of the sparse dual: v[col] += c * val * coef[r],
// one CTA per listed row (entries t, t + 256, ... of the row, four in
// flight; FP64 atomics).
__global__ void __launch_bounds__(256)
k_scatter_csr_rows(const long long* __restrict__ rowptr, const int* __restrict__ col,
                   const float* __restrict__ val, const int* __restrict__ idx,
                   long long nrows_total, long long ncols, const double* __restrict__ coef,
                   double c, double* __restrict__ v, unsigned* __restrict__ err) {
  pdl_wait();  // coef (the solve's Delta)
  pdl_trigger();
  const int r = blockIdx.x, tid = threadIdx.x;
  const long long row = idx[r];
  if (row < 0 || row >= nrows_total) {
    if (tid == 0) ca_flag(err, CA_DEV_ERR_ARG);
    return;
  }
  const double cr = c * coef[r];
  const long long e1 = rowptr[row + 1];
  for (long long eb = rowptr[row] + tid; eb < e1; eb += 4 * 256) {
    int fs[4];
    float vs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long e = eb + 256 * u;
      fs[u] = e < e1 ? col[e] : -1;
      vs[u] = e < e1 ? val[e] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (fs[u] >= 0 && fs[u] < ncols) atomicAdd(v + fs[u], (double)vs[u] * cr);
      else if (eb + 256 * u < e1) ca_flag(err, CA_DEV_ERR_ARG);
    }
  }
}

// Self-test of the bounded waits: thread 0 waits on an mbarrier that nothing
// arrives on; the wait gives up after limit_ns and flags CA_DEV_ERR_TIMEOUT.
__global__ void k_selftest_wait(unsigned long long limit_ns, unsigned* __restrict__ err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0u, err, limit_ns);
}

// G[i][j] = R[max(i,j)][min(i,j)] (full symmetric copy of the lower triangle)
__global__ void k_symmetrize(const double* __restrict__ R, int ldr, int sb, double* __restrict__ G) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)sb * sb) return;
  const int i = (int)(e / sb), j = (int)(e % sb);
  G[e] = i >= j ? R[(long long)i * ldr + j] : R[(long long)j * ldr + i];
}

// ---------------------------------------------------------------------------
// Host launchers of the templated kernels.
// ---------------------------------------------------------------------------
void launch_gram_simt(bool f64, dim3 grid, cudaStream_t st, const void* A, long long lda,
                      long long N, long long K, const int* idx, int sb, const double* v,
                      long long chunks_per_split, int sbp, double* part, double* ppart,
                      unsigned* err) {
  if (f64)
    k_gram_simt<double><<<grid, 256, 0, st>>>(static_cast<const double*>(A), lda, N, K, idx, sb, v,
                                              chunks_per_split, sbp, part, ppart, err);
  else
    k_gram_simt<float><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, N, K, idx, sb, v,
                                             chunks_per_split, sbp, part, ppart, err);
}

void launch_reduce(bool f32_partials, int grid, size_t smem, cudaStream_t st, const void* part,
                   const double* ppart, int P, int sbp, double* R, float2* Rs, double* pvec,
                   float2* Ginv, int ndiag, const SolveArgs& sa, unsigned* err) {
  if (f32_partials)
    k_reduce<float><<<grid, 256, smem, st>>>(static_cast<const float*>(part), ppart, P, sbp, R, Rs,
                                              pvec, Ginv, ndiag, sa, err);
  else
    k_reduce<double><<<grid, 256, smem, st>>>(static_cast<const double*>(part), ppart, P, sbp, R,
                                               Rs, pvec, Ginv, ndiag, sa, err);
}

template <typename K, typename... Args>
cudaError_t launch_programmatic(K kernel, unsigned grid, size_t smem, cudaStream_t st, Args... args);

void launch_chain(int b, size_t smem, cudaStream_t st, const float2* Rs, const double* pvec,
                  const float2* Ginv, const SolveArgs& sa, unsigned* err) {
  if (b <= 8)
    launch_programmatic(k_chain<8, 4>, 1u, smem, st, Rs, pvec, Ginv, sa, err);
  else if (b <= 16)
    launch_programmatic(k_chain<16, 3>, 1u, smem, st, Rs, pvec, Ginv, sa, err);
  else
    launch_programmatic(k_chain<32, 2>, 1u, smem, st, Rs, pvec, Ginv, sa, err);
}

template <typename K, typename... Args>
cudaError_t launch_programmatic(K kernel, unsigned grid, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int launch_reduce_chain(int grid, size_t smem, cudaStream_t st, const float* part,
                        const double* ppart, int P, int sbp, double* R, float2* Rs, double* pvec,
                        float2* Ginv, int ndiag, const SolveArgs& sa, unsigned* err,
                        unsigned* ticket) {
  cudaError_t e;
  if (sa.b <= 8)
    e = launch_programmatic(k_reduce_chain<float, 8, 4>, (unsigned)grid, smem, st, part, ppart, P,
                            sbp, R, Rs, pvec, Ginv, ndiag, sa, err, ticket);
  else if (sa.b <= 16)
    e = launch_programmatic(k_reduce_chain<float, 16, 3>, (unsigned)grid, smem, st, part, ppart, P,
                            sbp, R, Rs, pvec, Ginv, ndiag, sa, err, ticket);
  else
    e = cudaErrorInvalidValue;
  return (int)e;
}

// ---------------------------------------------------------------------------
// Stopping criterion (Sec. 5.1.5): the full residual of the current iterate,
// r = cP A v - cI x - cY y over all N rows of A, whose rows at the sampled
// indices are the right-hand side of each block subproblem.  Primal (A = X,
// v = rho = y - X^T w, x = w): (1/n) X rho - lambda w, the negative gradient
// of the objective; dual (A = X^T, v = w, x = alpha): X^T w - alpha - y, the
// dual residual up to its sign.
// ---------------------------------------------------------------------------

// q[r] += sum_k A[r][k] v[k] over the 32-column chunks [a0, a1) of this CTA's
// split (blockIdx.y); 8 warps x 8 rows per CTA, lane c takes column 32 a + c
// (a coalesced 128-byte row segment per load, panels or row-major).  FP32 A:
// exact products with the (hi, lo) FP32 split of v (FMA error terms) summed
// in double-float (v2 zero-padded to a multiple of 32); FP64 A: FP64.
// v and v2 change between calls (the solves update them): read through L2
// (ld.global.cg), never the non-coherent read-only path; A is constant.
// q starts at zero (k_residual_norm clears it after use).
template <typename T, bool PANEL>
__global__ void __launch_bounds__(256)
k_rowdot_dense(const T* __restrict__ A, long long lda, long long N, long long K,
               const double* __restrict__ v, const float2* __restrict__ v2,
               long long chunks_per_split, double* __restrict__ q) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)blockIdx.x * 64 + warp * 8;
  const long long natoms = (K + 31) / 32;
  const long long a0 = (long long)blockIdx.y * chunks_per_split;
  const long long a1 = min(natoms, a0 + chunks_per_split);
  if constexpr (sizeof(T) == 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long a = a0; a < a1; ++a) {
      const long long k = a * 32 + lane;
      const double vk = k < K ? __ldcg(v + k) : 0.0;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (r0 + j < N && k < K) acc[j] = fma((double)__ldg(A + (r0 + j) * lda + k), vk, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      double t = acc[j];
      for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0 && r0 + j < N) atomicAdd(q + r0 + j, t);
    }
  } else {
    float hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) hi[j] = lo[j] = 0.f;
    for (long long a = a0; a < a1; ++a) {
      const float2 vk = __ldcg(v2 + a * 32 + lane);
      const long long k = a * 32 + lane;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long r = r0 + j;
        float x = 0.f;
        if (r < N) {
          if constexpr (PANEL) x = __ldg(reinterpret_cast<const float*>(A) + (a * N + r) * 32 + lane);
          else if (k < K) x = __ldg(reinterpret_cast<const float*>(A) + r * lda + k);
        }
        df_dot_acc(x, vk.x, vk.y, hi[j], lo[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float2 t = df_norm(hi[j], lo[j]);
      for (int o = 16; o; o >>= 1)
        t = df_add(t, make_float2(__shfl_xor_sync(0xffffffffu, t.x, o),
                                  __shfl_xor_sync(0xffffffffu, t.y, o)));
      if (lane == 0 && r0 + j < N) atomicAdd(q + r0 + j, (double)t.x + (double)t.y);
    }
  }
}

// q[r] = (row r of the CSR matrix) . v, one warp per row, FP64 sums.
__global__ void __launch_bounds__(256)
k_rowdot_csr(const long long* __restrict__ rowptr, const int* __restrict__ col,
             const float* __restrict__ val, long long N, const double* __restrict__ v,
             double* __restrict__ q) {
  const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= N) return;
  double acc = 0.0;
  for (long long p = rowptr[r] + lane; p < rowptr[r + 1]; p += 32)
    acc = fma((double)val[p], __ldcg(v + col[p]), acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) q[r] = acc;
}

// *out += sum_r (cP q[r] - cI x[r] - cY y[r])^2 (FP64; y may be null), and
// q is cleared for the next use.
__global__ void __launch_bounds__(256)
k_residual_norm(double* __restrict__ q, const double* __restrict__ x, const double* __restrict__ y,
                long long N, double cP, double cI, double cY, double* __restrict__ out) {
  __shared__ double red[8];
  double acc = 0.0;
  for (long long r = (long long)blockIdx.x * 256 + threadIdx.x; r < N;
       r += (long long)gridDim.x * 256) {
    double t = cP * q[r] - cI * x[r];
    if (y) t -= cY * y[r];
    acc = fma(t, t, acc);
    q[r] = 0.0;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(out, t);
  }
}

void launch_residual(cudaStream_t st, int num_sms, const void* A, bool f64, bool panel,
                     long long lda, long long N, long long K, const double* v, const float2* v2,
                     const ca_csr_dev* csr, double* q, const double* x, const double* y,
                     double cP, double cI, double cY, double* out) {
  if (csr) {
    k_rowdot_csr<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(csr->rowptr, csr->col, csr->val, N, v, q);
  } else {
    const long long natoms = (K + 31) / 32, gx = (N + 63) / 64;
    const long long ys = std::max(1LL, std::min<long long>(natoms, (4LL * num_sms + gx - 1) / gx));
    const long long cps = (natoms + ys - 1) / ys;
    const dim3 grid((unsigned)gx, (unsigned)((natoms + cps - 1) / cps));
    if (f64)
      k_rowdot_dense<double, false><<<grid, 256, 0, st>>>(static_cast<const double*>(A), lda, N, K,
                                                         v, v2, cps, q);
    else if (panel)
      k_rowdot_dense<float, true><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, N, K, v,
                                                       v2, cps, q);
    else
      k_rowdot_dense<float, false><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, N, K,
                                                        v, v2, cps, q);
  }
  const long long rg = std::max(1LL, std::min<long long>((N + 255) / 256, 2LL * num_sms));
  k_residual_norm<<<(unsigned)rg, 256, 0, st>>>(q, x, y, N, cP, cI, cY, out);
}

void launch_sumsq(cudaStream_t st, int num_sms, double* q, const double* x, const double* y,
                  long long len, double cx, double cy, double* out) {
  const long long rg = std::max(1LL, std::min<long long>((len + 255) / 256, 2LL * num_sms));
  k_residual_norm<<<(unsigned)rg, 256, 0, st>>>(q, x, y, len, 0.0, -cx, -cy, out);
}

// Scaled FP16 Gram: for each row r of the N x K FP32 matrix A (row-major,
// leading dimension lda, or 32-column panels), the power of two
// rscale[r] = 2^(15 - e), where max_k |A[r][k]| = m 2^e with m in [0.5, 1):
// the row times rscale[r] has its largest magnitude in [2^14, 2^15), inside
// the FP16 range (largest finite 65504), and G_ij of the scaled rows is the
// true one times rscale[i] rscale[j] exactly.  A zero or non-finite row gets
// 1.  One warp per row.
__global__ void __launch_bounds__(256)
k_row_scale(const float* __restrict__ A, long long lda, long long N, long long K, int panel,
            float* __restrict__ rscale) {
  const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= N) return;
  float m[4] = {0.f, 0.f, 0.f, 0.f};
  if (panel) {  // element (r, 32 a + c) at A[(a N + r) 32 + c], zero past K
    const long long natoms = (K + 31) / 32;
#pragma unroll 4
    for (long long a = 0; a < natoms; ++a)
      m[a & 3] = fmaxf(m[a & 3], fabsf(__ldg(A + (a * N + r) * 32 + lane)));
  } else {
#pragma unroll 4
    for (long long k = lane; k < K; k += 32)
      m[(k >> 5) & 3] = fmaxf(m[(k >> 5) & 3], fabsf(__ldg(A + r * lda + k)));
  }
  float mx = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    float sc = 1.f;
    if (mx > 0.f && mx <= 3.4028234e38f) {
      int e = 0;
      frexpf(mx, &e);
      sc = ldexpf(1.f, min(max(15 - e, -120), 120));
    }
    rscale[r] = sc;
  }
}

void launch_row_scale(cudaStream_t st, const float* A, long long lda, long long N, long long K,
                      bool panel, float* rscale) {
  k_row_scale<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(A, lda, N, K, panel ? 1 : 0, rscale);
}

void launch_factor(cudaStream_t st, const double* R, const SolveArgs& sa, float2* Ginv,
                   unsigned* err) {
  k_factor<<<sa.s_cur, 256, 0, st>>>(R, sa, Ginv, err);
}

// Rs[j][i] = FP32 split of cG R[i][j] (transposed, as k_reduce writes it) for
// the lower-triangle entries outside the diagonal blocks (the sparse path

void launch_update_dense(bool f64, unsigned grid, size_t smem, cudaStream_t st, const void* A,
                         long long lda, long long N, long long K, const int* idx, int sb,
                         const double* delta, double cU, double* v, float2* v2, unsigned* err,
                         bool panel) {
  if (f64)
    k_update_dense<double, false><<<grid, 256, smem, st>>>(static_cast<const double*>(A), lda, N, K,
                                                            idx, sb, delta, cU, v, v2, err);
  else if (panel)
    k_update_dense<float, true><<<grid, 256, smem, st>>>(static_cast<const float*>(A), lda, N, K,
                                                          idx, sb, delta, cU, v, v2, err);
  else
    k_update_dense<float, false><<<grid, 256, smem, st>>>(static_cast<const float*>(A), lda, N, K,
                                                           idx, sb, delta, cU, v, v2, err);
}

void launch_recompute_dense(bool f64, dim3 grid, cudaStream_t st, const void* A, long long lda,
                            long long N, long long K, const double* x, const float2* x2, double c1,
                            long long rows_per_split, double* v, bool panel, const unsigned* nz) {
  if (f64)
    k_recompute_dense<double, false><<<grid, 256, 0, st>>>(static_cast<const double*>(A), lda, N, K,
                                                            x, x2, c1, rows_per_split, v, nz);
  else if (panel)
    k_recompute_dense<float, true><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, N, K, x,
                                                          x2, c1, rows_per_split, v, nz);
  else
    k_recompute_dense<float, false><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, N, K,
                                                           x, x2, c1, rows_per_split, v, nz);
}

// Repack a row-major N x K FP32 matrix (leading dimension lda, 16-byte aligned
// rows) into 32-column panels: P[(a N + r) 32 + c] = A[r][32 a + c], zero past
// K.  Units of 128 bytes (one row of one panel), 8 lanes each; consecutive
// units run along a row, so a warp reads 512 contiguous bytes and writes four
// full 128-byte lines.
__global__ void __launch_bounds__(256)
k_pack_panels(const float* __restrict__ A, long long N, long long K, long long lda,
              float* __restrict__ Pn) {
  const long long na = (K + 31) / 32;
  const long long units = N * na;
  const int q = threadIdx.x & 7;
  for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3; u < units;
       u += ((long long)gridDim.x * blockDim.x) >> 3) {
    const long long r = u / na, a = u - r * na;
    const long long k = a * 32 + 4 * q;
    const float* src = A + r * lda + k;
    float4 x;
    if (k + 4 <= K) {
      x = __ldg(reinterpret_cast<const float4*>(src));
    } else {
      x.x = k < K ? src[0] : 0.f;
      x.y = k + 1 < K ? src[1] : 0.f;
      x.z = k + 2 < K ? src[2] : 0.f;
      x.w = 0.f;
    }
    *reinterpret_cast<float4*>(Pn + (a * N + r) * 32 + 4 * q) = x;
  }
}

// Raise the dynamic shared-memory limit of the solve kernels to `bytes`, less
// each kernel's static shared memory (static + dynamic stays within the
// per-block maximum of the device).
template <typename K>
static cudaError_t set_dyn_smem(K kernel, int bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return e;
  const int cap = optin - (int)fa.sharedSizeBytes;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes < cap ? bytes : cap);
}

int launch_reduce_batch(int grid, cudaStream_t st, const RedInst* insts, const RedRole* roles,
                        unsigned* err) {
  return (int)launch_programmatic(k_reduce_batch, (unsigned)grid, 0, st, insts, roles, err);
}

int launch_chain_batch(int count, int bmax, size_t smem, cudaStream_t st, const RedInst* insts,
                       unsigned* err) {
  if (bmax <= 8)
    return (int)launch_programmatic(k_chain_batch<8, 4>, (unsigned)count, smem, st, insts, err);
  if (bmax <= 16)
    return (int)launch_programmatic(k_chain_batch<16, 3>, (unsigned)count, smem, st, insts, err);
  return (int)cudaErrorInvalidValue;
}

void launch_scatter_csr(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                        long long ncols, long long nlist, const double* coef, double c, double* v,
                        unsigned* err) {
  if (nlist <= 0) return;
  launch_programmatic(k_scatter_csr_rows, (unsigned)nlist, 0, st, csr.rowptr, csr.col, csr.val,
                      idx, nrows, ncols, coef, c, v, err);
}

void launch_csr_proj(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                     long long ncols, int sb, const double* w, double* pvec, unsigned* err) {
  if (sb <= 0) return;
  launch_programmatic(k_csr_proj, (unsigned)sb, 0, st, csr.rowptr, csr.col, csr.val, idx, nrows,
                      ncols, w, pvec, err);
}

void launch_csr_rownorm(cudaStream_t st, const ca_csr_dev& csr, long long nrows, double* rn) {
  if (nrows > 0)
    k_csr_rownorm<<<(unsigned)((nrows + 7) / 8), 256, 0, st>>>(csr.rowptr, csr.val, nrows, rn);
}

void launch_csr_prep(cudaStream_t st, int num_sms, const double* rn, long long nrows,
                     const double* G, const SolveArgs& sa, float2* Rs, float2* Ginv,
                     unsigned* err) {
  const long long conv = std::max(1LL, std::min<long long>(((long long)sa.sb * sa.sb + 255) / 256,
                                                           (long long)num_sms - 1));
  launch_programmatic(k_csr_prep, (unsigned)(sa.s_cur + conv), 0, st, rn, sa.idx, nrows, G, sa,
                      Rs, Ginv, err);
}

void launch_csr_gram(cudaStream_t st, int num_sms, const ca_csr_dev& csr, const int* idx,
                     long long nrows, long long ncols, int sb, int ldr, const double* w, double* G,
                     double* pvec, unsigned* err) {
  // q rows per tile: 32, halved while the tiles are fewer than two per SM
  auto count = [&](int qc) {
    int t = 0;
    for (int pb = 0; pb * kCsrPB < sb; ++pb) t += csr_tiles_of(pb, sb, qc);
    return t;
  };
  int qc = 32;
  while (qc > 1 && count(qc) < 2 * num_sms) qc >>= 1;
  launch_programmatic(k_csr_rows, (unsigned)((sb + 7) / 8), 0, st, csr.rowptr, csr.col, csr.val,
                      idx, nrows, ncols, sb, ldr, w, G, pvec, err);
  if (sb <= 1) return;
  if (sb <= 128) {  // few pairs: one warp per pair
    const long long npairs = (long long)sb * (sb - 1) / 2;
    launch_programmatic(k_csr_gram_pairs, (unsigned)std::max(1LL, (npairs + 7) / 8), 0, st,
                        csr.rowptr, csr.col, csr.val, idx, nrows, sb, ldr, G);
    return;
  }
  launch_programmatic(k_csr_gram, (unsigned)count(qc), kCsrSmem, st, csr.rowptr, csr.col,
                      csr.val, idx, nrows, ncols, sb, ldr, qc, w, G, pvec, err);
}

void launch_csr_prepare(cudaStream_t st, int num_sms, const ca_csr_dev& csr, long long nrows,
                        long long ncols, long long nnz, int* cnt, const int* dmap, int fd,
                        float* Xd, bool fill) {
  if (!fill) {
    const long long blocks = std::max(1LL, std::min<long long>((nnz + 255) / 256, 8LL * num_sms));
    k_colcount<<<(unsigned)blocks, 256, 0, st>>>(csr.col, nnz, ncols, cnt);
    return;
  }
  if (fd > 0)
    k_dense_fill<<<(unsigned)((nrows + 7) / 8), 256, 0, st>>>(csr.rowptr, csr.col, csr.val, nrows,
                                                                ncols, dmap, fd, Xd);
}

void launch_csr_rows(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                     long long ncols, int sb, int ldr, const double* w, double* G, double* pvec,
                     unsigned* err) {
  launch_programmatic(k_csr_rows, (unsigned)((sb + 7) / 8), 0, st, csr.rowptr, csr.col, csr.val,
                      idx, nrows, ncols, sb, ldr, w, G, pvec, err);
}

size_t csr_rangeoff_bytes(long long nrows, long long ncols) {
  return (size_t)nrows * (size_t)((ncols + kSgFR - 1) / kSgFR + 1) * sizeof(int);
}

void launch_csr_rangeoff(cudaStream_t st, const ca_csr_dev& csr, long long nrows, long long ncols,
                         int* roff) {
  if (nrows > 0)
    k_csr_rangeoff<<<(unsigned)((nrows + 7) / 8), 256, 0, st>>>(
        csr.rowptr, csr.col, nrows, (int)((ncols + kSgFR - 1) / kSgFR), roff);
}

void launch_csr_offdiag(cudaStream_t st, const ca_csr_dev& csr, const int* idx, long long nrows,
                        long long ncols, int sb, int ldr, double* G, const int* dmap,
                        const float* Xd, int fd, bool split, const int* roff) {
  if (sb <= 1) return;
  if (!split) {
    const long long npairs = (long long)sb * (sb - 1) / 2;
    launch_programmatic(k_csr_gram_pairs, (unsigned)std::max(1LL, (npairs + 7) / 8), 0, st,
                        csr.rowptr, csr.col, csr.val, idx, nrows, sb, ldr, G);
    return;
  }
  const int nb = (sb + kDgT - 1) / kDgT;
  launch_programmatic(k_dgram, (unsigned)(nb * (nb + 1) / 2), (size_t)2 * kDgT * (fd + 4) * 4, st,
                      Xd, fd, idx, sb, nrows, ldr, G);
  const int nr = (int)((ncols + kSgFR - 1) / kSgFR);
  launch_programmatic(k_sgram, (unsigned)nr, (size_t)kSgSmem, st, csr.rowptr, csr.col, csr.val,
                      idx, nrows, ncols, sb, dmap, ldr, G, roff, nr);
}

int launch_reduce_chain_f64(int grid, size_t smem, cudaStream_t st, const double* part,
                            const double* ppart, int sbp, double* R, float2* Rs, double* pvec,
                            float2* Ginv, int ndiag, const SolveArgs& sa, unsigned* err,
                            unsigned* ticket) {
  cudaError_t e;
  if (sa.b <= 8)
    e = launch_programmatic(k_reduce_chain<double, 8, 4>, (unsigned)grid, smem, st, part, ppart, 1,
                            sbp, R, Rs, pvec, Ginv, ndiag, sa, err, ticket);
  else if (sa.b <= 16)
    e = launch_programmatic(k_reduce_chain<double, 16, 3>, (unsigned)grid, smem, st, part, ppart, 1,
                            sbp, R, Rs, pvec, Ginv, ndiag, sa, err, ticket);
  else
    e = cudaErrorInvalidValue;
  return (int)e;
}

int set_solve_smem_limit(int bytes) {
  cudaError_t e[15] = {set_dyn_smem(k_solve, bytes), set_dyn_smem(k_csr_gram, kCsrSmem),
                      set_dyn_smem(k_sgram, kSgSmem),
                      set_dyn_smem(k_dgram, 2 * kDgT * (kCsrDenseMax + 4) * 4),
                      set_dyn_smem(k_chain<8, 4>, bytes),
                      set_dyn_smem(k_chain<16, 3>, bytes),
                      set_dyn_smem(k_chain<32, 2>, bytes),
                      set_dyn_smem(k_reduce<float>, bytes),
                      set_dyn_smem(k_reduce_chain<float, 8, 4>, bytes),
                      set_dyn_smem(k_reduce_chain<float, 16, 3>, bytes),
                      set_dyn_smem(k_reduce<double>, bytes),
                      set_dyn_smem(k_chain_batch<8, 4>, bytes),
                      set_dyn_smem(k_chain_batch<16, 3>, bytes),
                      set_dyn_smem(k_reduce_chain<double, 8, 4>, bytes),
                      set_dyn_smem(k_reduce_chain<double, 16, 3>, bytes)};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return (int)x;
  return 0;
}
