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
// With a fused update (s*b <= 128) each stage also brings in the previous
// outer step's rows: the loader warps apply that step's deferred update
// (v -= cU Yprev^T Delta, in double-float on the FP32-pair copy of v) to the
// stage's 32 columns, write it back, and project the current rows on the
// updated values: the update pass and the next Gram pass share one launch
// and one sweep over the K range.
// Every wait is bounded (CA_WAIT_LIMIT_NS) and raises CA_DEV_ERR_TIMEOUT.
#include "ca_kernels.cuh"

namespace {

constexpr int kLoaderWarps = 8;                      // 2 per SM sub-partition
constexpr int kLoaderThreads = 32 * kLoaderWarps;    // loaders / projection / epilogue
constexpr int kMmaWarp = kLoaderWarps;               // TMEM allocation and MMA issue
constexpr int kThreads = kLoaderThreads + 32;

template <int SBP, bool THREE, bool UPD = false>
struct TcCfg {
  static constexpr int kStageBytes = SBP * 128;                 // SBP rows x 32 fp32
  // [head tile | tail tile (3xTF32) | previous step's rows (fused update)]
  static constexpr int kStageTotal = kStageBytes * (1 + (THREE ? 1 : 0) + (UPD ? 1 : 0));
  static constexpr int kPrevOff = kStageBytes * (THREE ? 2 : 1);
  // ring depth: as many stages as fit (capped), so that short tiles (s*b <= 64)
  // still keep enough bytes in flight
  static constexpr int kNS = (176 * 1024) / kStageTotal < 32 ? (176 * 1024) / kStageTotal : 32;
  // SBP <= 128 with the 3-product split keeps two accumulators: D = hi hi^T
  // and T = hi lo^T (lo hi^T = T^T is added in the epilogue)
  static constexpr bool kSym = (SBP <= 128) && THREE;
  static constexpr int kTmemCols = (SBP == 256) ? 512 : (kSym ? 256 : 128);
  // the M = 128 MMA reads 128 rows of the head tile; with SBP < 128 the rows
  // past the tile are whatever follows in shared memory (their accumulator
  // rows are never stored), so keep that much slack past the ring
  static constexpr int kSlack = (SBP < 128 && kStageTotal < 16384) ? 16384 - kStageTotal : 0;
  static constexpr int kRPT = SBP / 32;                         // rows per loader thread
  // projection-vector ring: 2*NS slots of 32 (hi, lo) pairs, so that a slot is
  // rewritten only after every loader passed the barrier of a later stage
  static constexpr int kVRing = 2 * kNS * 256;
  // fused update: per-stage cross-group sums (16 x 32 FP32) and v_new split
  // per-warp column sums and the stage's updated v (fused update)
  static constexpr int kUpdBytes = UPD ? (kLoaderWarps * 32 * 4 + 32 * 8) : 0;
  // refill a stage after processing the current one (the empty-slot wait then
  // targets an MMA issued one iteration earlier); needs >= 4 stages
  static constexpr bool kLateRefill = kNS >= 4;
  static constexpr int kSmem = kNS * kStageTotal + kVRing + kUpdBytes + kSlack + 1024 + 512;
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

// Nearest TF32 value of x (ties away from zero), on the integer pipe: add
// half a TF32 unit in the last place to the magnitude bits, clear the 13
// low mantissa bits.  x - tf32_head(x) is exact in FP32.
__device__ __forceinline__ float tf32_head(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

template <int SBP, bool THREE, bool UPD>
__global__ void __launch_bounds__(kThreads, 1)
k_gram_tc(const float* __restrict__ A, long long lda, long long N, long long K,
          const int* __restrict__ idx, int sb, const float2* __restrict__ v2, long long natoms,
          float* __restrict__ part, double* __restrict__ ppart, unsigned* __restrict__ err,
          GramUpdate u) {
  using C = TcCfg<SBP, THREE, UPD>;
  constexpr int NS = C::kNS, RPT = C::kRPT;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stages = smem;  // NS x [big tile (| small tile)]
  unsigned char* vring = smem + NS * C::kStageTotal;  // 2*NS x 256 B
  float* ured = reinterpret_cast<float*>(vring + C::kVRing);  // [kLoaderWarps][32] (fused update)
  float2* vn2s = reinterpret_cast<float2*>(ured + kLoaderWarps * 32);  // [32]
  uint64_t* full = reinterpret_cast<uint64_t*>(vring + C::kVRing + C::kUpdBytes + C::kSlack);
  uint64_t* empty = full + NS;
  uint64_t* done = empty + NS;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x, P = gridDim.x;
  const long long a_begin = natoms * c / P, a_end = natoms * (c + 1) / P;
  const int T = (int)(a_end - a_begin);

  // Rows >= sb and columns >= K stay zero for the whole kernel.
  for (int e = tid; e < (NS * C::kStageTotal + C::kVRing + C::kUpdBytes + C::kSlack) / 16;
       e += kThreads)
    reinterpret_cast<uint4*>(stages)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], kLoaderThreads);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
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
  const int n1 = (SBP <= 128) ? ((sb + 31) & ~31) : 128;  // MMA N of the first (or only) tile
  const int n2 = (sb + 31) & ~31;                           // MMA N of rows 128..255 (SBP 256)

  if (warp < kLoaderWarps) {
    // ---------------- loaders / projection / epilogue ----------------
    const int g = tid >> 3, l = tid & 7;
    long long rowoff[RPT];
    uint32_t dsto[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int r = g + 32 * i;
      const long long gi = (r < sb) ? (long long)idx[r] : -1;
      const bool in_range = gi >= 0 && gi < N;
      if (r < sb && !in_range) ca_flag(err, CA_DEV_ERR_ARG);  // skipped, never read
      rowoff[i] = in_range ? gi * lda : -1;
      dsto[i] = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((l ^ (r & 7)) << 4));
    }
    // fused update: this thread's rows of the previous outer step and their
    // Delta as FP32 (hi, lo)
    const float2 u_cU2 = split_f64(u.cU);
    long long prevoff[UPD ? RPT : 1];
    float dph[UPD ? RPT : 1], dpl[UPD ? RPT : 1];
    if constexpr (UPD) {
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = g + 32 * i;
        const long long gi = (r < u.sb) ? (long long)u.idx[r] : -1;
        const bool in_range = gi >= 0 && gi < N;
        if (r < u.sb && !in_range) ca_flag(err, CA_DEV_ERR_ARG);
        prevoff[i] = in_range ? gi * lda : -1;
        const float2 d2 = split_f64(in_range ? u.delta[r] : 0.0);
        dph[i] = d2.x;
        dpl[i] = d2.y;
      }
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
      if constexpr (UPD) {
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          if (prevoff[i] >= 0)
            cp_async_16_zfill(dst + C::kPrevOff + dsto[i], A + prevoff[i] + (bytes ? k : 0), bytes);
      }
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
    auto refill = [&](int t) {  // stage t + NS - 1 into the slot of stage t - 1
      const int tn = t + NS - 1;
      if (ok && tn < T) {
        const int sn = tn % NS;
        if (tn >= NS) ok = mbar_wait_bounded(&empty[sn], (uint32_t)((tn / NS - 1) & 1), err);
        if (ok) issue(tn, sn);
      }
      cp_async_commit();
    };
    for (int t = 0; t < T; ++t) {
      if constexpr (C::kLateRefill) {
        cp_async_wait<NS - 2>();
      } else {
        refill(t);
        cp_async_wait<NS - 1>();
      }
      const int st = t % NS;
      unsigned char* big = stages + st * C::kStageTotal;
      if constexpr (!THREE) {  // the tile is ready for the MMA as loaded
        fence_proxy_async_smem();
        mbar_arrive(&full[st]);
      }
      // every loader's copies of this stage (incl. the v slice) have landed
      asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
      float vh[4], vl[4];
      if constexpr (UPD) {
        // deferred update of the previous outer step on this stage's 32
        // columns, v_new = v_old - cU * sum_r Yprev[r][k] Delta_r, in
        // double-float: per-thread sums over its rows, a shuffle over the 4
        // row groups of the warp, one shared-memory exchange between warps
        float up[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          if (prevoff[i] >= 0) {
            const float4 x = *reinterpret_cast<const float4*>(big + C::kPrevOff + dsto[i]);
            up[0] = fmaf(x.x, dph[i], fmaf(x.x, dpl[i], up[0]));
            up[1] = fmaf(x.y, dph[i], fmaf(x.y, dpl[i], up[1]));
            up[2] = fmaf(x.z, dph[i], fmaf(x.z, dpl[i], up[2]));
            up[3] = fmaf(x.w, dph[i], fmaf(x.w, dpl[i], up[3]));
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          up[e] += __shfl_xor_sync(0xffffffffu, up[e], 8);
          up[e] += __shfl_xor_sync(0xffffffffu, up[e], 16);
        }
        if (lane < 8)
          *reinterpret_cast<float4*>(ured + warp * 32 + 4 * l) =
              make_float4(up[0], up[1], up[2], up[3]);
        asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
        if (warp == 0) {  // lane = column: v_new once per column
          float sum = 0.f;
#pragma unroll
          for (int w2 = 0; w2 < kLoaderWarps; ++w2) sum += ured[32 * w2 + lane];
          const float2 vo = reinterpret_cast<const float2*>(vring + (t % (2 * NS)) * 256)[lane];
          const float2 vn = df_add(vo, df_neg(df_mul(u_cU2, make_float2(sum, 0.f))));
          vn2s[lane] = vn;
          const long long kk = (a_begin + t) * 32 + lane;
          if (kk < K) u.v2[kk] = vn;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 q = vn2s[4 * l + e];
          vh[e] = q.x;
          vl[e] = q.y;
        }
      } else {
        // projection vector slice as loaded (exact FP32 pairs)
        const float4* vs = reinterpret_cast<const float4*>(vring + (t % (2 * NS)) * 256 + l * 32);
        const float4 va = vs[0], vb = vs[1];
        vh[0] = va.x; vh[1] = va.z; vh[2] = vb.x; vh[3] = vb.z;
        vl[0] = va.y; vl[1] = va.w; vl[2] = vb.y; vl[3] = vb.w;
      }
      // projection on this thread's own chunks (exact FP32 inputs)
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
      if constexpr (C::kLateRefill) refill(t);  // stage t + NS - 1 into the slot of stage t - 1
    }
    cp_async_wait<0>();
    // projection partials: reduce over the 8 lanes sharing a row group
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      double s = (double)phi[i] + ((double)plo[i] + (double)pacc[i]);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      if (l == 0) ppart[(long long)c * SBP + g + 32 * i] = s;
    }
    // ---------------- epilogue: TMEM -> FP32 partial tiles ----------------
    mbar_wait_bounded(done, 0u, err);
    tc_fence_after();
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (= rows of the M = 128 tile)
    // and the 32-column chunks of parity w / 4
    const int lg = warp & 3, cpar = warp >> 2;
    const int trow = lg * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
    float* Pc = part + (long long)c * SBP * SBP;
    if constexpr (C::kSym) {
      // G = D + T + T^T: T goes through the (now idle) stage buffers as a
      // 128 x 129 FP32 array, read back transposed without bank conflicts
      float* Ts = reinterpret_cast<float*>(stages);
      for (int cc = 32 * cpar; cc < n1; cc += 64) {
        uint32_t r[32];
        tmem_ld32(tbase + 128u + (uint32_t)cc, r);
#pragma unroll
        for (int q = 0; q < 32; ++q) Ts[trow * 129 + cc + q] = __uint_as_float(r[q]);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kLoaderThreads) : "memory");
      for (int cc = 32 * cpar; cc < n1; cc += 64) {
        uint32_t r[32];
        tmem_ld32(tbase + (uint32_t)cc, r);
        if (cc <= trow && trow < SBP) {  // rows past a short tile hold garbage
          float4* dst = reinterpret_cast<float4*>(Pc + (long long)trow * SBP + cc);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int col = cc + 4 * q + e;
              o[e] = __uint_as_float(r[4 * q + e]) + Ts[trow * 129 + col] + Ts[col * 129 + trow];
            }
            dst[q] = make_float4(o[0], o[1], o[2], o[3]);
          }
        }
      }
    } else
    for (int cc = 32 * cpar; cc < n1; cc += 64) {  // rows 0..127, columns 0..n1-1
      uint32_t r[32];
      tmem_ld32(tbase + (uint32_t)cc, r);
      if (cc <= trow && trow < SBP) {  // rows past a short tile hold garbage
        float4* dst = reinterpret_cast<float4*>(Pc + (long long)trow * SBP + cc);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                               __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
      }
    }
    if constexpr (SBP == 256) {
      const int grow = 128 + trow;  // rows 128..255, columns 0..n2-1
      for (int cc = 32 * cpar; cc < n2; cc += 64) {
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
        if constexpr (C::kSym) {
          const uint64_t l0 = sw128_kmajor_desc(lb + kk * 32);
          mma_tf32(tmem + 128u, h0, l0, id1, acc);  // T = hi lo^T
        } else if constexpr (THREE) {
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
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)C::kTmemCols)
                 : "memory");
  }
}

template <int SBP, bool THREE, bool UPD>
int launch_one(const float* A, long long lda, long long N, long long K, const int* idx, int sb,
               const float2* v2, int P, float* part, double* ppart, unsigned* err,
               const GramUpdate& u, cudaStream_t stream) {
  using C = TcCfg<SBP, THREE, UPD>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<SBP, THREE, UPD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
    if (e != cudaSuccess) return (int)e;
    configured = true;
  }
  const long long natoms = (K + 31) / 32;
  k_gram_tc<SBP, THREE, UPD><<<P, kThreads, C::kSmem, stream>>>(A, lda, N, K, idx, sb, v2, natoms,
                                                                 part, ppart, err, u);
  return (int)cudaGetLastError();
}

}  // namespace

int gram_tc_max_sb() { return 256; }

int launch_gram_tc(const float* A, long long lda, long long N, long long K, const int* idx, int sb,
                   const float2* v2, int P, int sbp, float* part, double* ppart, unsigned* err,
                   int three_pass, cudaStream_t stream, const GramUpdate* upd) {
  const GramUpdate none{};
#define CA_TC_CASE(S, T, U, UU)                                                              \
  if (sbp == S && (three_pass != 0) == T)                                                  \
    return launch_one<S, T, U>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, UU, stream);
  if (upd && upd->sb > 0) {  // fused deferred update: s*b <= 128 only
    if (sbp > 128 || upd->sb > sbp) return (int)cudaErrorInvalidValue;
    CA_TC_CASE(32, true, true, *upd)
    CA_TC_CASE(32, false, true, *upd)
    CA_TC_CASE(64, true, true, *upd)
    CA_TC_CASE(64, false, true, *upd)
    CA_TC_CASE(128, true, true, *upd)
    CA_TC_CASE(128, false, true, *upd)
    return (int)cudaErrorInvalidValue;
  }
  CA_TC_CASE(32, true, false, none)
  CA_TC_CASE(32, false, false, none)
  CA_TC_CASE(64, true, false, none)
  CA_TC_CASE(64, false, false, none)
#undef CA_TC_CASE
  if (sbp == 128)
    return three_pass
               ? launch_one<128, true, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, none, stream)
               : launch_one<128, false, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, none, stream);
  if (sbp == 256)
    return three_pass
               ? launch_one<256, true, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, none, stream)
               : launch_one<256, false, false>(A, lda, N, K, idx, sb, v2, P, part, ppart, err, none, stream);
  return (int)cudaErrorInvalidValue;
}
