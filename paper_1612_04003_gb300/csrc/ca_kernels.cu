// ca_kernels.cu -- CUDA-core kernels of the CA-BCD / CA-BDCD outer step (sm_103a).
//
// Generic form used by every kernel here: A is an N x K row-major matrix whose
// rows are sampled (primal: A = X, N = d, K = n; dual: A = X^T, N = n, K = d),
// Y = the s'*b sampled rows of A, v the K-vector the Gram pass projects on
// (primal: rho = y - z with z = X^T w; dual: w).
#include "ca_kernels.cuh"

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
// the 64x64 tile (I, J), I >= J, of sum_{k in split c} Y[i][k] Y[j][k];
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
      P[(long long)(tI * 64 + ty * 4 + p) * sbp + (tJ * 64 + tx * 4 + q)] = acc[p][q];
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

// Reduce the split-K partials to R (lower triangle, FP64) and p, then the
// last CTA to finish runs the inner solves (no spin: a ticket counter).
template <typename PT>
__global__ void __launch_bounds__(256)
k_reduce_solve(const PT* __restrict__ part, const double* __restrict__ ppart, int P, int sbp,
               double* __restrict__ R, double* __restrict__ pvec, SolveArgs sa,
               unsigned* __restrict__ ticket, unsigned* __restrict__ err) {
  extern __shared__ double smem_d[];
  __shared__ bool is_last;
  const int sb = sa.sb;
  const long long nlow = (long long)sb * (sb + 1) / 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long sq = (long long)sbp * sbp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nlow + sb; e += stride) {
    if (e < nlow) {
      int i, j;
      tri_decode(e, i, j);
      const PT* src = part + (long long)i * sbp + j;
      double s = 0.0;
      for (int c = 0; c < P; ++c) s += (double)src[c * sq];
      R[(long long)i * sa.ldr + j] = s;
    } else {
      const int i = (int)(e - nlow);
      double s = 0.0;
      for (int c = 0; c < P; ++c) s += ppart[(long long)c * sbp + i];
      pvec[i] = s;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (threadIdx.x == 0) *ticket = 0u;
  block_solve(R, pvec, sa, err, smem_d);
}

template __global__ void k_reduce_solve<double>(const double*, const double*, int, int, double*,
                                                double*, SolveArgs, unsigned*, unsigned*);
template __global__ void k_reduce_solve<float>(const float*, const double*, int, int, double*,
                                               double*, SolveArgs, unsigned*, unsigned*);

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
// and sums over the rows, one FP64 subtraction per element.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_update_dense(const T* __restrict__ A, long long lda, long long N, long long K,
               const int* __restrict__ idx, int sb, const double* __restrict__ delta, double cU,
               double* __restrict__ v, unsigned* __restrict__ err) {
  extern __shared__ unsigned char smem_u[];
  int* sidx = reinterpret_cast<int*>(smem_u);
  double* sdl = reinterpret_cast<double*>(smem_u + ((sb * 4 + 255) & ~255));
  for (int r = threadIdx.x; r < sb; r += blockDim.x) {
    int gi = idx[r];
    double dl = delta[r];
    if (gi < 0 || (long long)gi >= N) {  // flagged; the row is skipped
      if (blockIdx.x == 0) ca_flag(err, CA_DEV_ERR_ARG);
      gi = 0;
      dl = 0.0;
    }
    sidx[r] = gi;
    sdl[r] = dl;
  }
  __syncthreads();
  const long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (k >= K) return;
  const int nk = (int)min(4ll, K - k);
  if constexpr (sizeof(T) == 8) {
    double acc[4] = {0, 0, 0, 0};
    for (int r = 0; r < sb; ++r) {
      const T* row = A + (long long)sidx[r] * lda + k;
      const double dl = sdl[r];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (e < nk) acc[e] = fma((double)row[e], dl, acc[e]);
    }
    for (int e = 0; e < nk; ++e) v[k + e] -= cU * acc[e];
  } else {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const bool vec = (nk == 4) && ((lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
#pragma unroll 8
    for (int r = 0; r < sb; ++r) {
      const float* row = reinterpret_cast<const float*>(A) + (long long)sidx[r] * lda + k;
      const double dl = sdl[r];
      const float dh = (float)dl, dlo = (float)(dl - (double)dh);
      float x[4];
      if (vec) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(row));
        x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = (e < nk) ? row[e] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] = fmaf(x[e], dh, fmaf(x[e], dlo, acc[e]));
    }
    for (int e = 0; e < nk; ++e) v[k + e] -= cU * (double)acc[e];
  }
}

template __global__ void k_update_dense<double>(const double*, long long, long long, long long,
                                                const int*, int, const double*, double, double*,
                                                unsigned*);
template __global__ void k_update_dense<float>(const float*, long long, long long, long long,
                                               const int*, int, const double*, double, double*,
                                               unsigned*);

// ---------------------------------------------------------------------------
// a6: full recompute  v[k] = c0 * y0[k] + c1 * sum_{r < N} A[r][k] x[r]
// (primal: rho = y - X^T w, or z = X^T w; dual: w = -X alpha/(lambda n)).
// Grid (K-blocks, row splits); row splits add into v with FP64 atomics after
// split 0 wrote the c0 * y0 term.  FP32 A: x split in two FP32 halves,
// FP32 sums over 32 rows, then FP64.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_recompute_dense(const T* __restrict__ A, long long lda, long long N, long long K,
                  const double* __restrict__ x, double c1, long long rows_per_split,
                  double* __restrict__ v) {
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
    const bool vec = (nk == 4) && ((lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    for (long long rb = r0; rb < r1; rb += 32) {
      float part[4] = {0.f, 0.f, 0.f, 0.f};
      const long long re = min(r1, rb + 32);
#pragma unroll 8
      for (long long r = rb; r < re; ++r) {
        const double xr = x[r];
        const float xh = (float)xr, xl = (float)(xr - (double)xh);
        const float* row = reinterpret_cast<const float*>(A) + r * lda + k;
        float q[4];
        if (vec) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(row));
          q[0] = t.x; q[1] = t.y; q[2] = t.z; q[3] = t.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) q[e] = (e < nk) ? row[e] : 0.f;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) part[e] = fmaf(q[e], xh, fmaf(q[e], xl, part[e]));
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] += (double)part[e];
    }
  }
  for (int e = 0; e < nk; ++e) atomicAdd(v + k + e, c1 * acc[e]);
}

template __global__ void k_recompute_dense<double>(const double*, long long, long long, long long,
                                                   const double*, double, long long, double*);
template __global__ void k_recompute_dense<float>(const float*, long long, long long, long long,
                                                  const double*, double, long long, double*);

// v = c0 * y0 (or 0 when y0 is null)
__global__ void k_axpby_init(const double* __restrict__ y0, double c0, long long K,
                             double* __restrict__ v) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) v[k] = y0 ? c0 * y0[k] : 0.0;
}

// ---------------------------------------------------------------------------
// Dual, sparse X (CSR of X^T, row i = column x_i of X, column indices sorted).
// ---------------------------------------------------------------------------
// a2+a3: R[p][q] = x_{I_p}^T x_{I_q} (q <= p) by sorted-list intersection,
// one warp per pair: lanes walk the shorter list and binary-search the longer.
__global__ void __launch_bounds__(256)
k_gram_csr(const long long* __restrict__ rowptr, const int* __restrict__ col,
           const float* __restrict__ val, const int* __restrict__ idx, long long nrows, int sb,
           int ldr, double* __restrict__ R, unsigned* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const long long npairs = (long long)sb * (sb + 1) / 2;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long e = warp; e < npairs; e += nwarps) {
    int p, q;
    tri_decode(e, p, q);
    const int ip = idx[p], iq = idx[q];
    if (ip < 0 || ip >= nrows || iq < 0 || iq >= nrows) {
      if (lane == 0) {
        ca_flag(err, CA_DEV_ERR_ARG);
        R[(long long)p * ldr + q] = 0.0;
      }
      continue;
    }
    long long a0 = rowptr[ip], a1 = rowptr[ip + 1];
    long long b0 = rowptr[iq], b1 = rowptr[iq + 1];
    if (a1 - a0 > b1 - b0) {
      long long t0 = a0, t1 = a1;
      a0 = b0; a1 = b1; b0 = t0; b1 = t1;
    }
    double s = 0.0;
    for (long long ea = a0 + lane; ea < a1; ea += 32) {
      const int f = col[ea];
      long long lo = b0, hi = b1;
      while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (col[mid] < f) lo = mid + 1; else hi = mid;
      }
      if (lo < b1 && col[lo] == f) s = fma((double)val[ea], (double)val[lo], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) R[(long long)p * ldr + q] = s;
  }
}

// p[r] = x_{I_r}^T w  (one warp per sampled column)
__global__ void __launch_bounds__(256)
k_proj_csr(const long long* __restrict__ rowptr, const int* __restrict__ col,
           const float* __restrict__ val, const int* __restrict__ idx, long long nrows,
           long long ncols, int sb, const double* __restrict__ w, double* __restrict__ pvec,
           unsigned* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= sb) return;
  const int ir = idx[r];
  if (ir < 0 || ir >= nrows) {
    if (lane == 0) {
      ca_flag(err, CA_DEV_ERR_ARG);
      pvec[r] = 0.0;
    }
    return;
  }
  const long long e0 = rowptr[ir], e1 = rowptr[ir + 1];
  double s = 0.0;
  for (long long e = e0 + lane; e < e1; e += 32) {
    const int f = col[e];
    if (f >= 0 && f < ncols) s = fma((double)val[e], w[f], s);
    else ca_flag(err, CA_DEV_ERR_ARG);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) pvec[r] = s;
}

// v[col] += c * val * coef[r] for the listed rows (a5 for CSR with coef =
// Delta alpha, c = -1/(lambda n); a6 with all rows, coef = alpha).
__global__ void __launch_bounds__(256)
k_scatter_csr(const long long* __restrict__ rowptr, const int* __restrict__ col,
              const float* __restrict__ val, const int* __restrict__ idx, long long nrows_total,
              long long ncols, long long nlist, const double* __restrict__ coef, double c,
              double* __restrict__ v, unsigned* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nlist) return;
  const long long row = idx ? (long long)idx[r] : r;
  if (row < 0 || row >= nrows_total) {
    if (lane == 0) ca_flag(err, CA_DEV_ERR_ARG);
    return;
  }
  const double cr = c * coef[r];
  for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
    const int f = col[e];
    if (f >= 0 && f < ncols) atomicAdd(v + f, (double)val[e] * cr);
    else ca_flag(err, CA_DEV_ERR_ARG);
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

void launch_reduce_solve_k(bool f32_partials, int grid, size_t smem, cudaStream_t st,
                           const void* part, const double* ppart, int P, int sbp, double* R,
                           double* pvec, const SolveArgs& sa, unsigned* ticket, unsigned* err) {
  if (f32_partials)
    k_reduce_solve<float><<<grid, 256, smem, st>>>(static_cast<const float*>(part), ppart, P, sbp,
                                                    R, pvec, sa, ticket, err);
  else
    k_reduce_solve<double><<<grid, 256, smem, st>>>(static_cast<const double*>(part), ppart, P,
                                                     sbp, R, pvec, sa, ticket, err);
}

void launch_update_dense(bool f64, unsigned grid, size_t smem, cudaStream_t st, const void* A,
                         long long lda, long long N, long long K, const int* idx, int sb,
                         const double* delta, double cU, double* v, unsigned* err) {
  if (f64)
    k_update_dense<double><<<grid, 256, smem, st>>>(static_cast<const double*>(A), lda, N, K, idx,
                                                     sb, delta, cU, v, err);
  else
    k_update_dense<float><<<grid, 256, smem, st>>>(static_cast<const float*>(A), lda, N, K, idx,
                                                    sb, delta, cU, v, err);
}

void launch_recompute_dense(bool f64, dim3 grid, cudaStream_t st, const void* A, long long lda,
                            long long N, long long K, const double* x, double c1,
                            long long rows_per_split, double* v) {
  if (f64)
    k_recompute_dense<double><<<grid, 256, 0, st>>>(static_cast<const double*>(A), lda, N, K, x, c1,
                                                     rows_per_split, v);
  else
    k_recompute_dense<float><<<grid, 256, 0, st>>>(static_cast<const float*>(A), lda, N, K, x, c1,
                                                    rows_per_split, v);
}

int set_solve_smem_limit(int bytes) {
  cudaError_t e1 = cudaFuncSetAttribute(k_reduce_solve<float>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaError_t e2 = cudaFuncSetAttribute(k_reduce_solve<double>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaError_t e3 = cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e1 != cudaSuccess) return (int)e1;
  if (e2 != cudaSuccess) return (int)e2;
  return (int)e3;
}
