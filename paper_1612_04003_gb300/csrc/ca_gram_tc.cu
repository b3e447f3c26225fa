// ca_gram_tc.cu -- the fused gather + Gram + projection pass on the sm_103a
// tensor cores (tcgen05, TF32 inputs, FP32 accumulation in tensor memory).
//
// One outer step of CA-BCD (Alg. 2) / CA-BDCD (Alg. 4) needs, from the s*b
// sampled rows Y of A (primal A = X; dual A = X^T), the Gram matrix Y Y^T and
// the projection Y v (primal v = y - z, dual v = w), both in one pass over Y
// ("compute the Gram matrix" of Alg. 2 / 4).  This kernel makes that pass:
//
//  * grid = P CTAs, one per SM; CTA c owns a contiguous range of 32-column
//    K-atoms and produces split-K partials (the single-GPU counterpart of the
//    paper's all-reduce of the Gram matrix, Sec. 4);
//  * warps 0-3 gather the sampled rows with 16-byte cp.async straight into
//    the 128-byte-swizzled K-major layout that tcgen05.mma reads (8-row atoms
//    of 1024 bytes, 16-byte chunk c of row r stored at chunk c ^ (r % 8)),
//    NS stages deep; the same warps form the projection from the staged tile
//    on CUDA cores (v split into two FP32 halves, FP32 products, FP64 sums);
//  * warp 4 allocates tensor memory and one thread issues the MMAs
//    (M = 128; N = the padded s*b) accumulating Y Y^T in TMEM;
//  * after the K loop warps 0-3 read TMEM (tcgen05.ld) and store the FP32
//    partial tile(s) that cover the lower triangle.
// With three_pass the FP32 inputs are split into a TF32 head and a TF32 tail
// (x = hi + lo) and hi*hi + hi*lo + lo*hi are accumulated (3xTF32).
// Every wait is bounded (CA_WAIT_LIMIT_NS) and raises CA_DEV_ERR_TIMEOUT.
#include "ca_kernels.cuh"

namespace {

constexpr int kLoaderThreads = 128;
constexpr int kThreads = 160;

template <int SBP, bool THREE>
struct TcCfg {
  static constexpr int kStageBytes = SBP * 128;                 // SBP rows x 32 fp32
  static constexpr int kStageTotal = THREE ? 2 * kStageBytes : kStageBytes;
  static constexpr int kNS = (192 * 1024) / kStageTotal;        // 12 / 6 / 6 / 3 stages
  static constexpr int kTmemCols = (SBP == 256) ? 512 : 128;
  static constexpr int kRPT = SBP / 16;                         // rows per loader thread
  // projection-vector ring: 2*NS slots of 32 (hi, lo) pairs, so that a slot is
  // rewritten only after every loader passed the barrier of a later stage
  static constexpr int kVRing = 2 * kNS * 256;
  static constexpr int kSmem = kNS * kStageTotal + kVRing + 1024 + 512;
};

__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  // tcgen05 shared-memory matrix descriptor: start address >> 4 (bits 0-13),
  // leading byte offset (unused for swizzled K-major, 16 B), stride byte
  // offset 1024 B between 8-row atoms (bits 32-45), fixed 0b001 at bits
  // 46-48, swizzle mode 2 = 128-byte swizzle (bits 61-63).
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1u << 16) |
         ((uint64_t)(1024u >> 4) << 32) | ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
  // kind::tf32 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = TF32
  // (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_head(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int SBP, bool THREE>
__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const float* __restrict__ A, long long lda, long long N, long long K,
          const int* __restrict__ idx, int sb, const float2* __restrict__ v2, long long natoms,
          float* __restrict__ part,
          double* __restrict__ ppart, unsigned* __restrict__ err) {
  using C = TcCfg<SBP, THREE>;
  constexpr int NS = C::kNS, RPT = C::kRPT;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stages = smem;  // NS x [big tile (| small tile)]
  unsigned char* vring = smem + NS * C::kStageTotal;  // 2*NS x 256 B
  uint64_t* full = reinterpret_cast<uint64_t*>(vring + C::kVRing);
  uint64_t* empty = full + NS;
  uint64_t* done = empty + NS;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x, P = gridDim.x;
  const long long a_begin = natoms * c / P, a_end = natoms * (c + 1) / P;
  const int T = (int)(a_end - a_begin);

  // Rows >= sb and columns >= K stay zero for the whole kernel.
  for (int e = tid; e < (NS * C::kStageTotal + C::kVRing) / 16; e += kThreads)
    reinterpret_cast<uint4*>(stages)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], kLoaderThreads);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"((uint32_t)C::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  const int n1 = (SBP == 128) ? ((sb + 31) & ~31) : 128;  // MMA N of the first (or only) tile
  const int n2 = (sb + 31) & ~31;                           // MMA N of rows 128..255 (SBP 256)

  if (warp < 4) {
    // ---------------- loaders / projection / epilogue ----------------
    const int g = tid >> 3, l = tid & 7;
    long long rowoff[RPT];
    uint32_t dsto[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = g + 16 * i;
      const long long gi = (r < sb) ? (long long)idx[r] : -1;
      const bool in_range = gi >= 0 && gi < N;
      if (r < sb && !in_range) ca_flag(err, CA_DEV_ERR_ARG);  // skipped, never read
      rowoff[i] = in_range ? gi * lda : -1;
      dsto[i] = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((l ^ (r & 7)) << 4));
    }
    const uint32_t stage0 = smem_u32(stages);
    const uint32_t vring0 = smem_u32(vring);
    auto issue = [&](int t, int slot) {
      const long long k = (a_begin + t) * 32 + 4 * l;
      const long long rem = K - k;
      const uint32_t bytes = rem >= 4 ? 16u : (rem > 0 ? (uint32_t)rem * 4u : 0u);
      const uint32_t dst = stage0 + (uint32_t)(slot * C::kStageTotal);
#pragma unroll
      for (int i = 0; i < RPT; ++i)
        if (rowoff[i] >= 0) cp_async_16_zfill(dst + dsto[i], A + rowoff[i] + (bytes ? k : 0), bytes);
      if (tid < 16)  // the stage's 32 (hi, lo) pairs of v (zero-padded to a multiple of 32)
        cp_async_16_zfill(vring0 + (uint32_t)((t % (2 * NS)) * 256 + tid * 16),
                          v2 + (a_begin + t) * 32 + 2 * tid, 16u);
    };
    // projection accumulators: FP32 partial sums over 8 stages, folded into
    // a compensated (hi, lo) FP32 pair
    float pacc[RPT], phi[RPT], plo[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      pacc[i] = 0.f;
      phi[i] = 0.f;
      plo[i] = 0.f;
    }
    bool ok = true;
    for (int t = 0; t < NS - 1; ++t) {
      if (t < T) issue(t, t);
      cp_async_commit();
    }
    for (int t = 0; t < T; ++t) {
      const int tn = t + NS - 1;
      if (ok && tn < T) {
        const int sn = tn % NS;
        if (tn >= NS) ok = mbar_wait_bounded(&empty[sn], (uint32_t)((tn / NS - 1) & 1), err);
        if (ok) issue(tn, sn);
      }
      cp_async_commit();
      cp_async_wait<NS - 1>();
      const int st = t % NS;
      unsigned char* big = stages + st * C::kStageTotal;
      if constexpr (!THREE) {  // the tile is ready for the MMA as loaded
        fence_proxy_async_smem();
        mbar_arrive(&full[st]);
      }
      // every loader's copies of this stage (incl. the v slice) have landed
      asm volatile("bar.sync 1, 128;" ::: "memory");
      // projection on this thread's own chunks (exact FP32 inputs)
      const float4* vs = reinterpret_cast<const float4*>(vring + (t % (2 * NS)) * 256 + l * 32);
      const float4 va = vs[0], vb = vs[1];
      const float vh[4] = {va.x, va.z, vb.x, vb.z};
      const float vl[4] = {va.y, va.w, vb.y, vb.w};
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        float4* p4 = reinterpret_cast<float4*>(big + dsto[i]);
        const float4 x = *p4;
        float a = pacc[i];
        a = fmaf(x.x, vh[0], fmaf(x.x, vl[0], a));
        a = fmaf(x.y, vh[1], fmaf(x.y, vl[1], a));
        a = fmaf(x.z, vh[2], fmaf(x.z, vl[2], a));
        a = fmaf(x.w, vh[3], fmaf(x.w, vl[3], a));
        pacc[i] = a;
        if constexpr (THREE) {
          const float4 h = make_float4(tf32_head(x.x), tf32_head(x.y), tf32_head(x.z), tf32_head(x.w));
          *p4 = h;
          *reinterpret_cast<float4*>(big + C::kStageBytes + dsto[i]) =
              make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
      }
      if ((t & 7) == 7) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          comp_add(phi[i], plo[i], pacc[i]);
          pacc[i] = 0.f;
        }
      }
      if constexpr (THREE) {  // head / tail tiles written: hand the stage to the MMA
        fence_proxy_async_smem();
        mbar_arrive(&full[st]);
      }
    }
    cp_async_wait<0>();
    // projection partials: reduce over the 8 lanes sharing a row group
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      double s = (double)phi[i] + ((double)plo[i] + (double)pacc[i]);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      if (l == 0) ppart[(long long)c * SBP + g + 16 * i] = s;
    }
    // ---------------- epilogue: TMEM -> FP32 partial tiles ----------------
    mbar_wait_bounded(done, 0u, err);
    tc_fence_after();
    const int trow = warp * 32 + lane;  // TMEM lane = row of the M = 128 tile
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
    float* Pc = part + (long long)c * SBP * SBP;
    for (int cc = 0; cc < n1; cc += 32) {  // rows 0..127, columns 0..n1-1
      uint32_t r[32];
      tmem_ld32(tbase + (uint32_t)cc, r);
      if (cc <= trow) {
        float4* dst = reinterpret_cast<float4*>(Pc + (long long)trow * SBP + cc);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                               __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
      }
    }
    if constexpr (SBP == 256) {
      const int grow = 128 + trow;  // rows 128..255, columns 0..n2-1
      for (int cc = 0; cc < n2; cc += 32) {
        uint32_t r[32];
        tmem_ld32(tbase + 128u + (uint32_t)cc, r);
        if (cc <= grow) {
          float4* dst = reinterpret_cast<float4*>(Pc + (long long)grow * SBP + cc);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                 __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
      }
    }
  } else if (lane == 0) {
    // ---------------- MMA issue (one thread) ----------------
    const uint32_t id1 = idesc_tf32(128, n1);
    const uint32_t id2 = idesc_tf32(128, n2);
    const uint32_t stage0 = smem_u32(stages);
    for (int t = 0; t < T; ++t) {
      const int st = t % NS;
      if (!mbar_wait_bounded(&full[st], (uint32_t)((t / NS) & 1), err)) break;
      tc_fence_after();
      const uint32_t hb = stage0 + (uint32_t)(st * C::kStageTotal);
      const uint32_t lb = hb + (uint32_t)C::kStageBytes;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t acc = (t > 0 || kk > 0) ? 1u : 0u;
        const uint64_t h0 = sw128_kmajor_desc(hb + kk * 32);
        mma_tf32(tmem, h0, h0, id1, acc);
        if constexpr (THREE) {
          const uint64_t l0 = sw128_kmajor_desc(lb + kk * 32);
          mma_tf32(tmem, h0, l0, id1, 1u);
          mma_tf32(tmem, l0, h0, id1, 1u);
        }
        if constexpr (SBP == 256) {
          const uint64_t h1 = sw128_kmajor_desc(hb + 16384 + kk * 32);
          mma_tf32(tmem + 128u, h1, h0, id2, acc);
          if constexpr (THREE) {
            const uint64_t l0 = sw128_kmajor_desc(lb + kk * 32);
            const uint64_t l1 = sw128_kmajor_desc(lb + 16384 + kk * 32);
            mma_tf32(tmem + 128u, h1, l0, id2, 1u);
            mma_tf32(tmem + 128u, l1, h0, id2, 1u);
          }
        }
      }
      mma_commit(&empty[st]);
    }
    mma_commit(done);
    // do not release tensor memory before the MMAs are complete
    mbar_wait_bounded(done, 0u, err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)C::kTmemCols)
                 : "memory");
  }
}

template <int SBP, bool THREE>
int launch_one(const float* A, long long lda, long long N, long long K, const int* idx, int sb,
               const float2* v2,
               int P, float* part, double* ppart, unsigned* err, cudaStream_t stream) {
  using C = TcCfg<SBP, THREE>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<SBP, THREE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return (int)e;
    configured = true;
  }
  const long long natoms = (K + 31) / 32;
  k_gram_tc<SBP, THREE><<<P, kThreads, C::kSmem, stream>>>(A, lda, N, K, idx, sb, v2, natoms, part,
                                                            ppart, err);
  return (int)cudaGetLastError();
}

}  // namespace

int gram_tc_max_sb() { return 256; }

int launch_gram_tc(const float* A, long long lda, long long N, long long K, const int* idx, int sb,
                   const float2* v2, int P, int sbp, float* part, double* ppart, unsigned* err,
                   int three_pass, cudaStream_t stream) {
  if (sbp == 128)
    return three_pass ? launch_one<128, true>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, stream)
                      : launch_one<128, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, stream);
  if (sbp == 256)
    return three_pass ? launch_one<256, true>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, stream)
                      : launch_one<256, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, stream);
  return (int)cudaErrorInvalidValue;
}
