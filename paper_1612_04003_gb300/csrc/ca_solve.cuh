// ca_solve.cuh -- device routines of step a4 (the s unrolled b x b solves of
// eq. "recur" and its dual analogue, Algorithms 2 and 4) shared by the
// kernels of ca_kernels.cu and the persistent solve of ca_persist.cu: the
// inversion of the diagonal blocks, the sums of split-K partials and the
// lookahead chain.
#pragma once
#include "ca_common.cuh"

// Gamma_j^{-1} for one b x b block by the Gauss-Jordan sweep operator on a
// symmetric positive definite matrix (Goodnight, 1979): sweeping pivot k maps
// a_kk -> -1/a_kk, a_ik -> a_ik/a_kk, a_kj -> a_kj/a_kk and
// a_ij -> a_ij - a_ik a_kj / a_kk; after all b pivots the matrix is -Gamma^{-1}.
// The sweep keeps the matrix symmetric, so pivot k needs only column k.  The
// CTA's 256 threads own one entry each (thread t: entries t + 256 q of the
// row-major b x b matrix, values a[q] in double-float); before pivot k the
// owners of column k publish it to shared memory (two buffers alternate: one
// barrier per pivot) and every thread forms 1 / a_kk from it.  Double-float on
// the FP32 pipe keeps the ~2^-44 accuracy at a fraction of the FP64 latency
// of this part.  NT = 256: every thread of the CTA calls this; NT = 64 (b <= 8,
// EPT = 1): two warps alone call it (warps 0-1, or the two warps whose
// threads pass their index 0..63 as tix) and the barrier per pivot is named
// barrier BAR over their 64 threads.
// Writes Gamma^{-1} (FP32 pairs, row-major) to out; a non-positive pivot
// raises CA_DEV_ERR_NOT_SPD.
template <int EPT, int NT = 256, int BAR = 1>
__device__ void cta_sweep_inverse(float2 (&a)[EPT], int b, float2* __restrict__ colbuf,
                                  float2* __restrict__ out, unsigned* __restrict__ err,
                                  int tix = -1) {
  static_assert(NT == 256 || NT == 64, "a CTA of 256 threads or two of its warps");
  const int t = tix >= 0 ? tix : (int)(threadIdx.x % NT);  // index among the NT threads
  int ri[EPT], ci[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = t + NT * q;
    ri[q] = e < b * b ? e / b : -1;
    ci[q] = e < b * b ? e - ri[q] * b : -1;
  }
  const bool active = t < b * b;
  for (int k = 0; k < b; ++k) {
    float2* ck = colbuf + (k & 1) * 33;  // [0, b): column k
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      if (ci[q] == k) {
        ck[ri[q]] = a[q];
        if (ri[q] == k && !(a[q].x > 0.f)) ca_flag(err, CA_DEV_ERR_NOT_SPD);
      }
    }
    if constexpr (NT == 64) asm volatile("bar.sync %0, 64;" ::"n"(BAR) : "memory");
    else __syncthreads();
    if (active) {
      // every thread forms 1 / a_kk itself (shorter than a broadcast)
      float2 d = ck[k];
      if (!(d.x > 0.f)) d = make_float2(1.f, 0.f);
      const float2 rd = df_rcp(d);
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int i = ri[q], j = ci[q];
        if (i < 0) continue;
        if (i == k && j == k) a[q] = df_neg(rd);
        else if (i == k) a[q] = df_mul(ck[j], rd);
        else if (j == k) a[q] = df_mul(ck[i], rd);
        else a[q] = df_add(a[q], df_neg(df_mul(df_mul(ck[i], rd), ck[j])));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q)
    if (ri[q] >= 0) out[t + NT * q] = df_neg(a[q]);
}

// Sum of the partials c = c0, c0 + step, ... < P of one entry (stride sq
// between partials), as a double-float value.  Up to U (FP32; FP64: U when
// U >= 32, else 16) loads are in flight at once (independent of the sums); FP32 partials are
// added in four compensated chains, FP64 partials by a pairwise FP64 tree.
template <typename PT, int U = 24>
__device__ __forceinline__ float2 sum_partials(const PT* __restrict__ src, int c0, int P, int step,
                                               long long sq) {
  static_assert(U % 4 == 0, "four compensated chains");
  if constexpr (sizeof(PT) == 4) {
    float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
    for (int base = c0; base < P; base += U * step) {
      float v[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {  // unconditional loads (clamped index), then select
        const int c = base + i * step;
        const float x = __ldcg(src + (long long)min(c, P - 1) * sq);
        v[i] = c < P ? x : 0.f;
      }
#pragma unroll
      for (int i = 0; i < U; ++i) comp_add(h[i & 3], l[i & 3], v[i]);
    }
    return df_add(df_add(df_norm(h[0], l[0]), df_norm(h[1], l[1])),
                  df_add(df_norm(h[2], l[2]), df_norm(h[3], l[3])));
  } else {
    constexpr int UD = U >= 32 ? U : 16;
    double acc = 0.0;
    for (int base = c0; base < P; base += UD * step) {
      double v[UD];
#pragma unroll
      for (int i = 0; i < UD; ++i) {
        const int c = base + i * step;
        const double x = __ldcg(src + (long long)min(c, P - 1) * sq);
        v[i] = c < P ? x : 0.0;
      }
      // pairwise tree over UD <= 128 values: at width w, v[i + w] folds onto
      // v[i] where it exists
      static_assert(UD <= 128, "tree depth");
#pragma unroll
      for (int w = 64; w >= 1; w /= 2)
#pragma unroll
        for (int i = 0; i < w; ++i)
          if (i + w < UD) v[i] += v[i + w];
      acc += v[0];
    }
    return split_f64(acc);
  }
}

// Sum of n double-float values by a balanced tree (n a power of two).
template <int N>
__device__ __forceinline__ float2 df_tree_sum(float2 (&v)[N]) {
  static_assert(N > 0 && (N & (N - 1)) == 0, "pairwise tree over a power of two");
#pragma unroll
  for (int w = N / 2; w >= 1; w /= 2)
#pragma unroll
    for (int i = 0; i < w; ++i) v[i] = df_add(v[i], v[i + w]);
  return v[0];
}

__device__ __forceinline__ float2 shfl_xor_df(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float2 shfl_df(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ void named_bar_sync(int id) {
  asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id) {
  asm volatile("bar.arrive %0, 256;" ::"r"(id) : "memory");
}

__device__ __forceinline__ void chain_cta_sync() {
  asm volatile("bar.sync 6, 256;" ::: "memory");
}

// The dependent chain with lookahead (one CTA of 256 threads; b <= BMAX <= 16,
// sb <= 256), from Rs (cG-scaled, transposed), p and the diagonal-block
// inverses Ginv.  Warp 0 runs only the dependent path: for step j it forms
// Delta_j = Gamma_j^{-1} rb_j (BMAX x BMAX products over 32 lanes, shuffle
// sums), publishes it, folds it into the b rows of block j+1 and adds the
// sums the other warps kept for those rows, which gives rb_{j+1}.  Warps 1-7
// fold each published Delta_j into the rows >= (j+2) b (two rows per
// thread), hand over the sums of the rows of block j+2, and stream the Rs
// columns of later steps through a shared-memory ring (16-byte cp.async.cg
// copies of row pairs, slot layout [q][row]).  Warp 0 and the others meet at
// named barriers, two per step alternating by parity (D: Delta_j published;
// F: the folds of step j done), so neither waits for a full-CTA barrier.  The
// index-overlap term cI [I_r = I_t] Delta_t (eq. "recur" and its dual
// analogue) is added where the sampled indices coincide.  All arithmetic on
// the dependent path is double-float; FP64 converts in and out.  Only warps
// 0-7 of the CTA take part (CTA-wide steps use named barrier 6 over 256
// threads), so a larger CTA may give its other warps other work.  With a
// ticket the chain first waits (bounded) until *ticket >= nready; the count
// is cleared afterwards unless reset_ticket is false (a count that keeps
// growing across outer steps).
template <int BMAX, int DEPTH>
__device__ void chain_la_body(const float2* __restrict__ Rs, const double* __restrict__ pvec,
                              const float2* __restrict__ Ginv, const SolveArgs& a,
                              unsigned* __restrict__ err, double* smem_d,
                              unsigned* __restrict__ ticket = nullptr, unsigned nready = 0,
                              bool reset_ticket = true) {
  static_assert(BMAX == 8 || BMAX == 16, "lookahead chain: BMAX 8 or 16");
  constexpr int LPR = 32 / BMAX, CPL = BMAX / LPR;  // warp 0: lanes per row, columns per lane
  constexpr unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = a.b, sb = a.sb, ldr = a.ldr, s = a.s_cur;
  float2* ring = reinterpret_cast<float2*>(smem_d);     // DEPTH x BMAX x 256
  float2* Gs = ring + (size_t)DEPTH * BMAX * 256;       // sb*b: Gamma_j^{-1}
  float2* rhs0s = Gs + (size_t)sb * b;                   // 256: cP p - cI x0 - cY y
  float2* dall = rhs0s + 256;                            // 256: all Delta
  float2* accb = dall + 256;                             // [2][16]: sums handed to warp 0
  float2* ovlb = accb + 32;                              // [2][16]: overlap sums
  int* sidx = reinterpret_cast<int*>(ovlb + 32);         // 256
  const uint32_t ring0 = smem_u32(ring);
  const bool ld_ok = (ldr & 1) == 0;  // 16-byte row pairs need an even leading dimension
  if (!ld_ok && tid == 0) ca_flag(err, CA_DEV_ERR_ARG);
  const int cu = tid - 32;  // index among warps 1-7
  auto fetch = [&](int j) {  // warps 1-7: columns jb .. jb+b of rows >= jb + b, slot j % DEPTH
    const int jb = j * b;
    if (j < s && ld_ok) {
      const int p0 = (jb + b) >> 1, np = ((sb + 1) >> 1) - p0;
      for (int u = cu; u < b * np; u += 224) {
        const int q = u / np, pr = 2 * (p0 + u - q * np);
        cp_async_16_zfill(ring0 + 8u * (uint32_t)(((j % DEPTH) * BMAX + q) * 256 + pr),
                          Rs + (long long)(jb + q) * ldr + pr, 16u);
      }
    }
    cp_async_commit();
  };
  // the sampled indices and x0, y there do not depend on the reduction
  double xy = 0.0;  // -cI x0[I] - cY y[I]
  if (tid < sb) {
    const int gi = a.idx[tid];
    if (gi >= 0 && gi < a.N) {
      xy = -a.cI * __ldcg(a.x + gi);
      if (a.yv) xy -= a.cY * a.yv[gi];
    } else {
      ca_flag(err, CA_DEV_ERR_ARG);
    }
    sidx[tid] = gi;
  }
  if (ticket) {  // the reducing CTAs of this grid: R, Rs, p and Ginv complete
    if (tid == 0) {
      const uint64_t t0 = ca_globaltimer();
      // gives up after the limit, or at once when another wait of the
      // grid has already given up
      for (uint32_t it = 1; *(volatile unsigned*)ticket < nready; ++it) {
        if ((it & 255u) == 0u) {
          if (*(volatile unsigned*)err & CA_DEV_ERR_TIMEOUT) break;
          if (ca_globaltimer() - t0 > CA_WAIT_LIMIT_NS) {
            ca_flag(err, CA_DEV_ERR_TIMEOUT);
            break;
          }
        }
      }
      if (reset_ticket) *ticket = 0u;  // for the next launch (which starts after this grid ends)
      __threadfence();
    }
    chain_cta_sync();
  }
  if (warp > 0)
    for (int d = 0; d < DEPTH - 1; ++d) fetch(d);
  for (int e = tid; e < sb * b; e += 256) Gs[e] = __ldcg(Ginv + e);
  if (tid < sb) rhs0s[tid] = split_f64(a.cP * __ldcg(pvec + tid) + xy);
  if (warp > 0) cp_async_wait<DEPTH - 2>();  // step 0's columns
  chain_cta_sync();
  const float2 cI2 = split_f64(a.cI);
  const float2 z2 = make_float2(0.f, 0.f);
  if (warp == 0) {
    const int i = lane / LPR, c0 = (lane % LPR) * CPL;
    float2 rbv = i < b ? rhs0s[i] : z2;  // rb of the current block, row i
    for (int j = 0; j < s; ++j) {
      const int jb = j * b;
      float2 pr[CPL];
#pragma unroll
      for (int cc = 0; cc < CPL; ++cc) {
        const int c = c0 + cc;
        const float2 rbc = shfl_df(rbv, c * LPR);
        pr[cc] = (i < b && c < b) ? df_mul(Gs[(size_t)j * b * b + i * b + c], rbc) : z2;
      }
      float2 dl = df_tree_sum(pr);
#pragma unroll
      for (int o = LPR / 2; o >= 1; o /= 2) dl = df_add(dl, shfl_xor_df(dl, o));
      if (i < b && (lane % LPR) == 0) dall[jb + i] = dl;
      __syncwarp();
      named_bar_arrive(2 + (j & 1));  // D(j): Delta_j published
      if (j + 1 < s) {
        if (j >= 1) named_bar_sync(4 + ((j - 1) & 1));  // F(j-1): sums of block j+1, columns of step j
        const int rowp = (j + 1) * b + i;
        const bool rv = i < b && rowp < sb;
        const int gp = rv ? sidx[rowp] : -2;
        const float2* slot = ring + (size_t)(j % DEPTH) * BMAX * 256;
        float2 u[CPL];
        float2 ov = z2;
        bool hit = false;
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
          const int c = c0 + cc;
          const float2 dc = shfl_df(dl, c * LPR);
          u[cc] = z2;
          if (rv && c < b) {
            u[cc] = df_mul(slot[c * 256 + rowp], dc);
            if (sidx[jb + c] == gp) {
              ov = df_add(ov, dc);
              hit = true;
            }
          }
        }
        float2 us = df_tree_sum(u);
#pragma unroll
        for (int o = LPR / 2; o >= 1; o /= 2) us = df_add(us, shfl_xor_df(us, o));
        if (__any_sync(FULL, hit)) {
#pragma unroll
          for (int o = LPR / 2; o >= 1; o /= 2) ov = df_add(ov, shfl_xor_df(ov, o));
        }
        const int hb = ((j + 1) & 1) * 16 + i;
        const float2 accv = (j >= 1 && rv) ? accb[hb] : z2;
        const float2 ovv = (j >= 1 && rv) ? ovlb[hb] : z2;
        rbv = rv ? df_add(rhs0s[rowp], df_neg(df_add(df_add(accv, us), df_mul(cI2, df_add(ovv, ov)))))
                 : z2;
      }
    }
  } else {
    const int r1 = cu, r2 = cu + 224;
    const int g1 = r1 < sb ? sidx[r1] : -2, g2 = r2 < sb ? sidx[r2] : -2;
    float2 acc1 = z2, acc2 = z2, ov1 = z2, ov2 = z2;
    for (int j = 0; j < s; ++j) {
      const int jb = j * b, lo = (j + 2) * b;
      named_bar_sync(2 + (j & 1));  // D(j)
      const float2* slot = ring + (size_t)(j % DEPTH) * BMAX * 256;
      float2 dq[BMAX];
      int iq[BMAX];
#pragma unroll
      for (int q = 0; q < BMAX; ++q) {
        dq[q] = q < b ? dall[jb + q] : z2;
        iq[q] = q < b ? sidx[jb + q] : -3;
      }
      auto fold = [&](int r, int g, float2& acc, float2& ov) {
        float2 pr[BMAX];
        unsigned m = 0;
#pragma unroll
        for (int q = 0; q < BMAX; ++q) {
          pr[q] = q < b ? df_mul(slot[q * 256 + r], dq[q]) : z2;
          m |= (iq[q] == g) ? (1u << q) : 0u;
        }
        acc = df_add(acc, df_tree_sum(pr));
        while (m) {  // sampled index shared with an earlier row (rare)
          const int q = __ffs(m) - 1;
          ov = df_add(ov, dall[jb + q]);
          m &= m - 1;
        }
      };
      if (r1 >= lo && r1 < sb) fold(r1, g1, acc1, ov1);
      if (r2 >= lo && r2 < sb) fold(r2, g2, acc2, ov2);
      const int hb = ((j + 2) & 1) * 16;
      if (r1 >= lo && r1 < lo + b && r1 < sb) {
        accb[hb + r1 - lo] = acc1;
        ovlb[hb + r1 - lo] = ov1;
      }
      if (r2 >= lo && r2 < lo + b && r2 < sb) {
        accb[hb + r2 - lo] = acc2;
        ovlb[hb + r2 - lo] = ov2;
      }
      fetch(j + DEPTH - 1);        // into the slot of step j-1 (warp 0 is done with it)
      cp_async_wait<DEPTH - 2>();  // this thread's columns of step j+1 have landed
      if (j + 2 < s) named_bar_arrive(4 + (j & 1));  // F(j)
    }
    cp_async_wait<0>();
  }
  chain_cta_sync();
  if (tid < sb) {  // Delta out, x += Delta (atomic: an index may recur across blocks)
    const float2 d2 = dall[tid];
    const double dv = (double)d2.x + (double)d2.y;
    if (!isfinite(dv)) ca_flag(err, CA_DEV_ERR_NONFINITE);
    a.delta[tid] = dv;
    const int g = sidx[tid];
    if (g >= 0 && g < a.N) atomicAdd(a.x + g, dv);
  }
}

