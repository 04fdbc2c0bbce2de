// Shared-memory FFT engine and the generic FFT pass kernel.
//
// Every pass reads the sequences it transforms from contiguous memory: a CTA loads B
// sequences of length L (a supported length of fft_core.cuh; register-staged, 16 complex values
// per thread, 32 at L = 8192, all loads in flight before the first shared-memory store), runs the Stockham stages of fft_core.cuh
// on them in shared memory (sequence b at b * LP, element i at spad(i)), and hands them to the
// pass's store, which writes either along the sequence (row-major) or across the B sequences
// (transposed: consecutive threads write consecutive sequences of one output index). The
// transposed store is how a pass produces the layout the next pass reads contiguously, so no
// pass ever reads a column.
#pragma once
#include "fr_internal.cuh"

namespace fr {

constexpr int pow2_floor(int x) { return x < 2 ? 1 : 2 * pow2_floor(x / 2); }

// Pass configuration of length LEN at P points per thread (16; 32 for the ops that ask for it
// at L = 8192, see op_pts).
template <int LEN, int P = 16>
struct FftCfg {
  static_assert(fft_length_ok(LEN), "unsupported FFT length");
  static_assert(P == 16 || P == 32, "16 or 32 points per thread");
  static constexpr int L = LEN;
  // L >= 8192 runs one sequence per CTA so that two CTAs share an SM and overlap their load,
  // transform and store phases; 4096 <= L < 8192 keeps two (16-byte transposed stores)
  static constexpr int B = (L >= 8192) ? 1 : (L >= 4096 ? 2 : pow2_floor(4096 / L));
  static constexpr int PTS = P;
  static constexpr int NT = (B * L) / PTS;
  static constexpr int LP = spad_len(L) + 1;  // odd stride between sequences
  static constexpr size_t SMEM = size_t(B) * LP * sizeof(float2);
  // CTAs per SM the register budget is sized for: four at L = 2048 (64 registers, no spills);
  // never fewer than 64 registers a thread (the 640- and 768-thread CTAs of 5 2^k and 3 2^k)
  static constexpr int FIT64 = 65536 / (NT * 64) > 1 ? 65536 / (NT * 64) : 1;
  static constexpr int cap(int m) { return m < FIT64 ? m : FIT64; }
  // the 3 2^k and 5 2^k lengths (160- to 768-thread CTAs) target 64 registers outright
  // (measured 18 % faster at 1536 than the power-of-two rule, which let 110 registers through)
  static constexpr bool POW2 = (L & (L - 1)) == 0;
  // 32 points a thread hold 64 registers of data alone: two CTAs per SM (128 registers)
  static constexpr int MINB = PTS == 32 ? 2
                              : POW2    ? cap(NT >= 1024 ? 1 : (NT >= 512 || L < 2048 ? 2 : 4))
                                        : FIT64;
  static constexpr int MINB_SUM = PTS == 32 ? 1 : cap(NT >= 512 ? 1 : 2);  // multi-output passes
  // two-transform passes; the mixed lengths one CTA below the 64-register count (measured
  // fastest at 1280 and 1536: 72 and 80 registers, small spills)
  static constexpr int MINB_TWO = PTS == 32 ? 2
                                  : POW2    ? cap(NT >= 1024 ? 1 : 2)
                                            : (FIT64 > 1 ? FIT64 - 1 : 1);
};

// Stage twiddles w^(r k) of a power-of-two length: w^k = exp(DIR 2 pi i k tstep / L) from one
// sincospif (the argument 2 k tstep / L is exact in FP32), its powers w^(k 2^e) by squaring and
// the others by products (twiddle_rec), so no stage waits on a table load; other lengths load
// their twiddles from the table (apply_twiddles).
// Bulk L2 prefetch of a contiguous range: one instruction, no registers held, nothing to wait
// for. The instruction takes a 16-byte aligned address and a multiple of 16 bytes; other ranges
// (rows of images whose side is not a multiple of 4) are left alone.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  if ((((uintptr_t)p) & 15) != 0 || (bytes & 15) != 0 || bytes == 0) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// A pass's CTAs start in index order, about two per SM at a time: the CTA PF_AHEAD indices on
// starts roughly when this one ends, so this one prefetches that CTA's input into L2.
constexpr int PF_AHEAD = 2 * 152;

template <int L, int R, int DIR>
__device__ __forceinline__ void stage_twiddles(float2* v, const float2* __restrict__ tw, int k,
                                               int tstep) {
  if constexpr ((L & (L - 1)) == 0 && (R & (R - 1)) == 0) {
    constexpr int LB = ilog2(R);
    float2 pw[LB];
    float sn, cs;
    sincospif((float)(2 * k * tstep) * (1.f / (float)L), &sn, &cs);
    pw[0] = make_float2(cs, DIR < 0 ? -sn : sn);
#pragma unroll
    for (int e = 1; e < LB; ++e) pw[e] = cmul(pw[e - 1], pw[e - 1]);
    float2 wr[R];
    twiddle_rec<R, 1>(v, pw, wr);
  } else {
    apply_twiddles<R, DIR>(v, tw, k, tstep);
  }
}

template <int L, int ST, int DIR, int P = 16>
__device__ __forceinline__ void fft_stages(float2* s, const float2* __restrict__ tw) {
  if constexpr (ST < fft_num_stages(L, P)) {
    using C = FftCfg<L, P>;
    constexpr int B = C::B, NT = C::NT, LP = C::LP;
    constexpr int R = fft_radix(L, ST, P);
    constexpr int NS = fft_ns_before(L, ST, P);
    constexpr int LR = L / R;
    constexpr int NTASK = B * LR;
    // power-of-two radices split evenly (16 / R tasks per thread); radix 3 and 5 take
    // ceil(16 / R) with the last round partly idle
    constexpr bool EVEN = NTASK % NT == 0;
    constexpr int TPT = (NTASK + NT - 1) / NT;
    constexpr int TSTEP = L / (NS * R);
    float2 v[TPT][R];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int t = threadIdx.x + q * NT;
      if (EVEN || t < NTASK) {
        const int b = t / LR, j = t % LR;
        const int k = (NS & (NS - 1)) == 0 ? (j & (NS - 1)) : j % NS;
        const float2* src = s + b * LP;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = src[spad(j + r * LR)];
        if constexpr (ST > 0) stage_twiddles<L, R, DIR>(v[q], tw, k, TSTEP);
        dft_r<R, DIR>(v[q]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int t = threadIdx.x + q * NT;
      if (EVEN || t < NTASK) {
        const int b = t / LR, j = t % LR;
        const int k = (NS & (NS - 1)) == 0 ? (j & (NS - 1)) : j % NS;
        float2* dst = s + b * LP;
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[spad(base + r * NS)] = v[q][r];
      }
    }
    __syncthreads();
    fft_stages<L, ST + 1, DIR, P>(s, tw);
  }
}

// The first stage of the power-of-two lengths whose schedule opens with a radix equal to the
// points per thread P (16, or 32 at 8192) runs on the values a thread loaded itself: thread t
// takes sequence b = t / (L/P) and task j = t % (L/P), loads x[j + k L/P] (k < P, consecutive
// threads on consecutive elements), transforms them in registers and writes the stage's
// outputs, so that stage costs no shared-memory round trip and no barrier. Other lengths load
// idx = t + k NT (sequence idx / L, element idx % L) and run every stage in shared memory.
template <int L, int P = 16>
constexpr bool fuse_first() {
  using C = FftCfg<L, P>;
  return C::POW2 && fft_radix(L, 0, P) == P && C::B * L / C::NT == P;
}

// sequence (within the CTA) and element of the k-th value a thread loads
template <int L, int P = 16>
__device__ __forceinline__ void load_pos(int k, int* b, int* i) {
  if constexpr (fuse_first<L, P>()) {
    constexpr int Q = L / P;
    *b = threadIdx.x / Q;
    *i = threadIdx.x % Q + k * Q;
  } else {
    const int idx = threadIdx.x + k * FftCfg<L, P>::NT;
    *b = idx / L;
    *i = idx % L;
  }
}

// The transform of the loaded values r (load_pos order) into shared memory, in natural order;
// `landed` runs once every thread's values are in shared memory (before the remaining stages).
template <int L, int DIR, int P = 16, class F>
__device__ __forceinline__ void fft_from_regs(float2* s, float2* r, const float2* __restrict__ tw,
                                              F landed) {
  using C = FftCfg<L, P>;
  if constexpr (fuse_first<L, P>()) {
    constexpr int Q = L / P;
    const int b = threadIdx.x / Q, j = threadIdx.x % Q;
    float2 v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = r[k];
    dft_r<P, DIR>(v);
    float2* dst = s + b * C::LP;
#pragma unroll
    for (int k = 0; k < P; ++k) dst[spad(P * j + k)] = v[k];
    __syncthreads();
    landed();
    fft_stages<L, 1, DIR, P>(s, tw);
  } else {
    constexpr int PER = C::B * L / C::NT;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + k * C::NT;
      s[(idx / L) * C::LP + spad(idx % L)] = r[k];
    }
    __syncthreads();
    landed();
    fft_stages<L, 0, DIR, P>(s, tw);
  }
}

// Points per thread of an op's pass at length L: the two-transform passes at 8192 (forward,
// pointwise product, inverse in one CTA) run 32 (three stages per transform; measured 25 %
// faster than four), everything else 16 (twice the resident warps for the latency of the
// loads, measured faster for the single-transform passes).
template <int L, class Op>
constexpr int op_pts() {
  return (Op::TWO && L == 8192) ? 32 : 16;
}

// The same stages, except that the last one hands its outputs to sink(b, i, value) (sequence b
// of the CTA, output index i in natural order) instead of writing them back to shared memory:
// its task j of sequence b produces outputs i = j + r L/R, so consecutive threads hold
// consecutive outputs and a row-major store from the sink is coalesced. Saves the last
// shared-memory round trip and its two barriers. Shared memory is left as the stage read it.
template <int L, int ST, int DIR, int P, class Sink>
__device__ __forceinline__ void fft_stages_direct(float2* s, const float2* __restrict__ tw,
                                                  Sink sink) {
  constexpr int S = fft_num_stages(L, P);
  if constexpr (ST < S - 1) {
    using C = FftCfg<L, P>;
    constexpr int B = C::B, NT = C::NT, LP = C::LP;
    constexpr int R = fft_radix(L, ST, P);
    constexpr int NS = fft_ns_before(L, ST, P);
    constexpr int LR = L / R;
    constexpr int NTASK = B * LR;
    constexpr bool EVEN = NTASK % NT == 0;
    constexpr int TPT = (NTASK + NT - 1) / NT;
    constexpr int TSTEP = L / (NS * R);
    float2 v[TPT][R];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int t = threadIdx.x + q * NT;
      if (EVEN || t < NTASK) {
        const int b = t / LR, j = t % LR;
        const int k = (NS & (NS - 1)) == 0 ? (j & (NS - 1)) : j % NS;
        const float2* src = s + b * LP;
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = src[spad(j + r * LR)];
        if constexpr (ST > 0) stage_twiddles<L, R, DIR>(v[q], tw, k, TSTEP);
        dft_r<R, DIR>(v[q]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int t = threadIdx.x + q * NT;
      if (EVEN || t < NTASK) {
        const int b = t / LR, j = t % LR;
        const int k = (NS & (NS - 1)) == 0 ? (j & (NS - 1)) : j % NS;
        float2* dst = s + b * LP;
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[spad(base + r * NS)] = v[q][r];
      }
    }
    __syncthreads();
    fft_stages_direct<L, ST + 1, DIR, P>(s, tw, sink);
  } else if constexpr (ST == S - 1) {
    using C = FftCfg<L, P>;
    constexpr int B = C::B, NT = C::NT, LP = C::LP;
    constexpr int R = fft_radix(L, ST, P);
    constexpr int NS = fft_ns_before(L, ST, P);
    constexpr int LR = L / R;
    static_assert(NS * R == L && NS == LR, "last stage");
    constexpr int NTASK = B * LR;
    constexpr bool EVEN = NTASK % NT == 0;
    constexpr int TPT = (NTASK + NT - 1) / NT;
    // one task at a time: the sink's work per output stays out of the other task's registers
#pragma unroll 1
    for (int q = 0; q < TPT; ++q) {
      const int t = threadIdx.x + q * NT;
      if (EVEN || t < NTASK) {
        const int b = t / LR, j = t % LR;
        const float2* src = s + b * LP;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[spad(j + r * LR)];
        if constexpr (ST > 0) stage_twiddles<L, R, DIR>(v, tw, j, 1);
        dft_r<R, DIR>(v);
#pragma unroll
        for (int r = 0; r < R; ++r) sink(b, j + r * LR, v[r]);
      }
    }
  }
}

// Each (sequence, output index) pair that fft_stages_direct hands to the sink, for this thread,
// in the same order: f(b, i) for the thread's tasks of the last stage.
template <int L, int P, class F>
__device__ __forceinline__ void for_direct_outputs(F f) {
  using C = FftCfg<L, P>;
  constexpr int S = fft_num_stages(L, P);
  constexpr int R = fft_radix(L, S - 1, P);
  constexpr int LR = L / R, NT = C::NT;
  constexpr int NTASK = C::B * LR;
  constexpr bool EVEN = NTASK % NT == 0;
  constexpr int TPT = (NTASK + NT - 1) / NT;
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int t = threadIdx.x + q * NT;
    if (EVEN || t < NTASK) {
      const int b = t / LR, j = t % LR;
#pragma unroll
      for (int r = 0; r < R; ++r) f(b, j + r * LR);
    }
  }
}

// fft_from_regs whose last stage goes to sink(b, i, value) (fft_stages_direct)
template <int L, int DIR, int P = 16, class F, class Sink>
__device__ __forceinline__ void fft_from_regs_direct(float2* s, float2* r,
                                                     const float2* __restrict__ tw, F landed,
                                                     Sink sink) {
  using C = FftCfg<L, P>;
  if constexpr (fuse_first<L, P>()) {
    constexpr int Q = L / P;
    const int b = threadIdx.x / Q, j = threadIdx.x % Q;
    float2 v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = r[k];
    dft_r<P, DIR>(v);
    float2* dst = s + b * C::LP;
#pragma unroll
    for (int k = 0; k < P; ++k) dst[spad(P * j + k)] = v[k];
    __syncthreads();
    landed();
    fft_stages_direct<L, 1, DIR, P>(s, tw, sink);
  } else {
    constexpr int PER = C::B * L / C::NT;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + k * C::NT;
      s[(idx / L) * C::LP + spad(idx % L)] = r[k];
    }
    __syncthreads();
    landed();
    fft_stages_direct<L, 0, DIR, P>(s, tw, sink);
  }
}

// Read-only view of one sequence in shared memory.
struct SeqView {
  const float2* p;
  __device__ __forceinline__ float2 operator[](int i) const { return p[spad(i)]; }
};

// Transposed stores write each output index o as a run of consecutive sequences. With few
// sequences per CTA that run is short (8 bytes at B = 1), so ops that support it (Op::GROUP)
// gather the run of a thread-block cluster instead: at B = 1, CL = 4 CTAs hold 4 consecutive
// sequences, and after a cluster barrier each CTA writes 1/CL of the outputs as 32-byte groups,
// reading the other CTAs' sequences through distributed shared memory (8 sequences in 64-byte
// groups measured slower). Such ops add
//   float2 pick(int seq, int o, SeqView v)            the value store() would write
//   void store_group(int seq0, int o, const float2* v, int n)   n <= 4 consecutive sequences
constexpr int GROUP_SEQ = 4;  // consecutive sequences per output run (32 bytes)

template <int B, class Op>
constexpr int cluster_size() {
  // one sequence per CTA (8192 and 16384 points); at B = 2 the 16-byte runs measured as fast
  if constexpr (Op::TRANSPOSED && Op::GROUP && B == 1) return GROUP_SEQ;
  return 1;
}

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// generic address of the same shared-memory location in cluster CTA `rank`
__device__ __forceinline__ const float2* cluster_map(const float2* p, uint32_t rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"((uint64_t)p), "r"(rank));
  return reinterpret_cast<const float2*>(out);
}

// Generic pass. blockIdx.x selects B consecutive sequences, blockIdx.y an image (ops that batch
// images use it); ops with SEQ_Y swap the two, so that the CTAs of one sequence block for all
// images run next to each other and share the block's input through L2. Op provides:
//   static constexpr bool TRANSPOSED   store mapping (see above)
//   static constexpr bool TWO          second transform (DIR2) after mid()
//   int nseq() const, int nout() const      (host and device)
//   float2 load(int seq, int i)        element i of the sequence (zero padding costs no load)
//   void after_load(int seq0, int nb)  after every thread's loads have landed
//   void mid(float2* s, int seq0)      between the transforms (TWO)
//   double store(int seq, int o, SeqView v)   o < nout(); per-thread results are summed
//   void finish(int seq0, double acc)
template <int LEN, int DIR, int DIR2, class Op>
__global__ void __launch_bounds__(FftCfg<LEN, op_pts<LEN, Op>()>::NT,
                                  Op::TWO ? FftCfg<LEN, op_pts<LEN, Op>()>::MINB_TWO
                                          : FftCfg<LEN, op_pts<LEN, Op>()>::MINB)
    fft_pass_kernel(Op op, const float2* __restrict__ tw) {
  constexpr int P = op_pts<LEN, Op>();
  using C = FftCfg<LEN, P>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  constexpr int PER = B * L / NT;
  extern __shared__ float2 smem[];
  const int nseq = op.nseq();
  const int seq0 = (Op::SEQ_Y ? blockIdx.y : blockIdx.x) * B;
  if constexpr (Op::PREFETCH) {
    // SEQ_Y passes start the CTAs of all images of one sequence block together
    const int ahead = Op::SEQ_Y ? (PF_AHEAD + (int)gridDim.x - 1) / (int)gridDim.x : PF_AHEAD;
    if (threadIdx.x < B && seq0 + ahead * B + (int)threadIdx.x < nseq)
      op.prefetch(seq0 + ahead * B + threadIdx.x);
  }
  float2 r[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int b, i;
    load_pos<L, P>(k, &b, &i);
    r[k] = (seq0 + b < nseq) ? op.load(seq0 + b, i) : make_float2(0.f, 0.f);
  }
  if constexpr (Op::DIRECT && !Op::TWO && !Op::TRANSPOSED) {
    // row-major outputs straight from the last stage
    double dacc = 0.0;
    fft_from_regs_direct<L, DIR, P>(
        smem, r, tw, [&] { if (seq0 < nseq) op.after_load(seq0, min(B, nseq - seq0)); },
        [&](int b, int i, float2 v) {
          if (seq0 + b < nseq) dacc += op.direct(seq0 + b, i, v);
        });
    op.finish(seq0, dacc);
    return;
  }
  fft_from_regs<L, DIR, P>(smem, r, tw, [&] {
    if (seq0 < nseq) op.after_load(seq0, min(B, nseq - seq0));
  });
  if constexpr (Op::TWO) {
    op.template mid<B, NT, L, LP>(smem, seq0);
    __syncthreads();
    fft_stages<L, 0, DIR2, P>(smem, tw);
  }
  const int nout = op.nout();
  double acc = 0.0;
  constexpr int CL = cluster_size<B, Op>();
  if constexpr (CL > 1) {
    // every CTA of the cluster has transformed its sequences: gather 4 per output index
    cluster_barrier();
    const uint32_t rank = cluster_rank();
    const int g0 = seq0 - (int)rank * B;  // first sequence of the cluster
    const int per = (nout + CL - 1) / CL;
    const int o0 = (int)rank * per, o1 = min(nout, o0 + per);
    const int n = min(CL * B, nseq - g0);
    if (n > 0) {
      const float2* views[CL];
#pragma unroll
      for (int c = 0; c < CL; ++c) views[c] = cluster_map(smem, (uint32_t)c);
      for (int o = o0 + threadIdx.x; o < o1; o += NT) {
        float2 v[CL * B];
#pragma unroll
        for (int c = 0; c < CL; ++c)
#pragma unroll
          for (int b = 0; b < B; ++b) {
            const int q = c * B + b;
            v[q] = q < n ? op.pick(g0 + q, o, SeqView{views[c] + b * LP}) : make_float2(0.f, 0.f);
          }
        op.store_group(g0, o, v, n);
      }
    }
    cluster_barrier();  // the other CTAs have read this CTA's shared memory
  } else if constexpr (Op::TRANSPOSED) {
    for (int idx = threadIdx.x; idx < B * nout; idx += NT) {
      const int o = idx / B, b = idx % B;
      if (seq0 + b < nseq) acc += op.store(seq0 + b, o, SeqView{smem + b * LP});
    }
  } else {
    for (int idx = threadIdx.x; idx < B * nout; idx += NT) {
      const int b = idx / nout, o = idx % nout;
      if (seq0 + b < nseq) acc += op.store(seq0 + b, o, SeqView{smem + b * LP});
    }
  }
  op.finish(seq0, acc);
}

template <int LEN, int DIR, int DIR2, class Op>
int launch_pass(const Op& op, int nimg, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LEN, op_pts<LEN, Op>()>;
  const int nblk = (op.nseq() + C::B - 1) / C::B;
  if (nblk == 0 || nimg == 0) return FR_OK;
  auto kern = fft_pass_kernel<LEN, DIR, DIR2, Op>;
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  constexpr int CL = cluster_size<C::B, Op>();
  if constexpr (CL > 1) {
    // whole clusters: the CTAs past the last sequence transform zeros and store nothing
    cudaLaunchConfig_t cfg = {};
    const unsigned nb = (nblk + CL - 1) / CL * CL;
    cfg.gridDim = Op::SEQ_Y ? dim3(nimg, nb) : dim3(nb, nimg);
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = Op::SEQ_Y ? 1 : CL;
    at[0].val.clusterDim.y = Op::SEQ_Y ? CL : 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FR_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, op, tw));
  } else {
    kern<<<Op::SEQ_Y ? dim3(nimg, nblk) : dim3(nblk, nimg), C::NT, C::SMEM, s>>>(op, tw);
  }
  FR_LAUNCHED();
  return FR_OK;
}

// Multi-input pass: op.ntrans() transforms per sequence, each of its own input, whose outputs
// are combined per output element and written once (row-major mapping; blockIdx.x selects B
// sequences). The last stage of every transform hands its outputs to the combination directly
// (fft_stages_direct); each output's running sum sits in shared memory after the sequences, in
// a slot only the thread holding that output ever touches.
//   Trans trans(int t)                              transform t's parameters
//   float2 load(const Trans&, int seq, int i)       element i of its input
//   int out_of(int i)                               output of transform index i, or -1
//   float term(const Trans&, int seq, int o, float2 z)   its contribution to output o
//   void store(int seq, int o, float acc)
// Outputs per sequence nout() <= L / 2.
template <int LEN, int DIR, class Op>
__global__ void __launch_bounds__(FftCfg<LEN>::NT, FftCfg<LEN>::MINB)
    fft_pass_accum_kernel(Op op, const float2* __restrict__ tw) {
  using C = FftCfg<LEN>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  constexpr int PER = B * L / NT;
  constexpr int HALF = L / 2;
  extern __shared__ float2 smem[];
  float* acc = reinterpret_cast<float*>(smem + B * LP);  // [B][L / 2]
  const int nseq = op.nseq(), ntr = op.ntrans();
  const int seq0 = blockIdx.x * B;
  if constexpr (Op::PREFETCH) {
    if (threadIdx.x < B && seq0 + PF_AHEAD * B + (int)threadIdx.x < nseq)
      op.prefetch(seq0 + PF_AHEAD * B + threadIdx.x);
  }
  for_direct_outputs<L, 16>([&](int b, int i) {
    const int o = op.out_of(i);
    if (o >= 0) acc[b * HALF + o] = 0.f;
  });
#pragma unroll 1
  for (int t = 0; t < ntr; ++t) {
    const typename Op::Trans tp = op.trans(t);
    if (t > 0) __syncthreads();  // the previous transform's last stage has read its inputs
    float2 r[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      int b, i;
      load_pos<L>(k, &b, &i);
      r[k] = (seq0 + b < nseq) ? op.load(tp, seq0 + b, i) : make_float2(0.f, 0.f);
    }
    fft_from_regs_direct<L, DIR>(smem, r, tw, [] {}, [&](int b, int i, float2 z) {
      const int o = op.out_of(i);
      if (o >= 0 && seq0 + b < nseq) acc[b * HALF + o] += op.term(tp, seq0 + b, o, z);
    });
  }
  for_direct_outputs<L, 16>([&](int b, int i) {
    const int o = op.out_of(i);
    if (o >= 0 && seq0 + b < nseq) op.store(seq0 + b, o, acc[b * HALF + o]);
  });
}

template <int LEN, int DIR, class Op>
int launch_pass_accum(const Op& op, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LEN>;
  const int nblk = (op.nseq() + C::B - 1) / C::B;
  if (nblk == 0) return FR_OK;
  auto kern = fft_pass_accum_kernel<LEN, DIR, Op>;
  constexpr size_t smem = C::SMEM + (size_t)C::B * LEN / 2 * sizeof(float);
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  kern<<<nblk, C::NT, smem, s>>>(op, tw);
  FR_LAUNCHED();
  return FR_OK;
}

// Multi-output pass: one load per element, then op.nterms() transforms of inputs derived from it
// (blockIdx.x selects B sequences):
//   float2 load(int seq, int i)        raw element (zero padding costs no load)
//   float2 prep(int t, float2& raw)    input of transform t; may update raw for transform t + 1
//   double store(int t, int seq, int o, SeqView v)   mapping per Op::TRANSPOSED
template <int LEN, int DIR, class Op>
__global__ void __launch_bounds__(FftCfg<LEN>::NT, FftCfg<LEN>::MINB_SUM)
    fft_pass_multi_kernel(Op op, const float2* __restrict__ tw) {
  using C = FftCfg<LEN>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  constexpr int PER = B * L / NT;
  extern __shared__ float2 smem[];
  const int nseq = op.nseq(), nout = op.nout(), nterm = op.nterms();
  const int seq0 = blockIdx.x * B;
  float2 r[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int b, i;
    load_pos<L>(k, &b, &i);
    r[k] = (seq0 + b < nseq) ? op.load(seq0 + b, i) : make_float2(0.f, 0.f);
  }
  for (int t = 0; t < nterm; ++t) {
    if (t > 0) __syncthreads();  // the previous transform's outputs have been read
    float2 x[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) x[k] = op.prep(t, r[k]);
    fft_from_regs<L, DIR>(smem, x, tw, [] {});
    if constexpr (Op::TRANSPOSED) {
      for (int idx = threadIdx.x; idx < B * nout; idx += NT) {
        const int o = idx / B, b = idx % B;
        if (seq0 + b < nseq) op.store(t, seq0 + b, o, SeqView{smem + b * LP});
      }
    } else {
      for (int idx = threadIdx.x; idx < B * nout; idx += NT) {
        const int b = idx / nout, o = idx % nout;
        if (seq0 + b < nseq) op.store(t, seq0 + b, o, SeqView{smem + b * LP});
      }
    }
  }
}

template <int LEN, int DIR, class Op>
int launch_pass_multi(const Op& op, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LEN>;
  const int nblk = (op.nseq() + C::B - 1) / C::B;
  if (nblk == 0) return FR_OK;
  auto kern = fft_pass_multi_kernel<LEN, DIR, Op>;
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  kern<<<nblk, C::NT, C::SMEM, s>>>(op, tw);
  FR_LAUNCHED();
  return FR_OK;
}

// group store helper: n <= GROUP_SEQ consecutive complex values at dst (16-byte vector stores
// when the group is whole and aligned)
__device__ __forceinline__ void store_run(float2* dst, const float2* v, int n) {
  if (n == GROUP_SEQ && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
    for (int g = 0; g < GROUP_SEQ; g += 2)
      reinterpret_cast<float4*>(dst)[g / 2] = make_float4(v[g].x, v[g].y, v[g + 1].x, v[g + 1].y);
  } else {
    for (int g = 0; g < n; ++g) dst[g] = v[g];
  }
}

// a[t] of a small parameter array with every index static (no copy of the array to local memory)
template <class T, int N>
__device__ __forceinline__ T pick_static(const T (&a)[N], int t) {
  T r = a[0];
#pragma unroll
  for (int k = 1; k < N; ++k)
    if (t == k) r = a[k];
  return r;
}

// Defaults for the optional parts of an op.
struct OpBase {
  static constexpr bool TRANSPOSED = false;
  static constexpr bool TWO = false;
  static constexpr bool GROUP = false;
  static constexpr bool SEQ_Y = false;
  // row-major ops with DIRECT provide double direct(int seq, int i, float2 value): the store of
  // transform output i (natural order), called once per output from the last stage; the
  // returned values are summed per thread for finish() as store()'s are
  static constexpr bool DIRECT = false;
  __device__ void after_load(int, int) const {}
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2*, int) const {}
  __device__ void finish(int, double) const {}
  // ops with PREFETCH provide void prefetch(int seq): L2 prefetches of that sequence's input
  static constexpr bool PREFETCH = false;
  __device__ void prefetch(int) const {}
};


// Dispatch a templated functor (templated on the length) on a runtime log2 length in [5, 14].
#define FR_LOG2_DISPATCH(log2l, F, ...)                      \
  switch (log2l) {                                           \
    case 5: return F<32>(__VA_ARGS__);                       \
    case 6: return F<64>(__VA_ARGS__);                       \
    case 7: return F<128>(__VA_ARGS__);                      \
    case 8: return F<256>(__VA_ARGS__);                      \
    case 9: return F<512>(__VA_ARGS__);                      \
    case 10: return F<1024>(__VA_ARGS__);                    \
    case 11: return F<2048>(__VA_ARGS__);                    \
    case 12: return F<4096>(__VA_ARGS__);                    \
    case 13: return F<8192>(__VA_ARGS__);                    \
    case 14: return F<16384>(__VA_ARGS__);                   \
    default:                                                 \
      ::fr::set_error("FFT length 2^%d unsupported", log2l); \
      return FR_EUNSUPPORTED;                                \
  }

// Dispatch on a runtime length: the powers of two 32 .. 16384, 3 2^k for 48 .. 6144 and
// 5 2^k for 80 .. 5120 (the reduced-padding PSF transforms of images up to 4096 a side);
// fft_len_supported() agrees.
#define FR_LEN_CASES(F, ...)                      \
  case 32: return F<32>(__VA_ARGS__);             \
  case 64: return F<64>(__VA_ARGS__);             \
  case 128: return F<128>(__VA_ARGS__);           \
  case 256: return F<256>(__VA_ARGS__);           \
  case 512: return F<512>(__VA_ARGS__);           \
  case 1024: return F<1024>(__VA_ARGS__);         \
  case 2048: return F<2048>(__VA_ARGS__);         \
  case 4096: return F<4096>(__VA_ARGS__);         \
  case 8192: return F<8192>(__VA_ARGS__);         \
  case 16384: return F<16384>(__VA_ARGS__);       \
  case 48: return F<48>(__VA_ARGS__);             \
  case 96: return F<96>(__VA_ARGS__);             \
  case 192: return F<192>(__VA_ARGS__);           \
  case 384: return F<384>(__VA_ARGS__);           \
  case 768: return F<768>(__VA_ARGS__);           \
  case 1536: return F<1536>(__VA_ARGS__);         \
  case 3072: return F<3072>(__VA_ARGS__);         \
  case 6144: return F<6144>(__VA_ARGS__);         \
  case 80: return F<80>(__VA_ARGS__);             \
  case 160: return F<160>(__VA_ARGS__);           \
  case 320: return F<320>(__VA_ARGS__);           \
  case 640: return F<640>(__VA_ARGS__);           \
  case 1280: return F<1280>(__VA_ARGS__);         \
  case 2560: return F<2560>(__VA_ARGS__);         \
  case 5120: return F<5120>(__VA_ARGS__);

#define FR_LEN_DISPATCH(len, F, ...)                            \
  switch (len) {                                                \
    FR_LEN_CASES(F, __VA_ARGS__)                                \
    default:                                                    \
      ::fr::set_error("FFT length %d unsupported", (int)(len)); \
      return FR_EUNSUPPORTED;                                   \
  }

// The noise passes transform the unpadded image, so they also take the image sides whose odd
// part has several factors 3 and 5: c 2^k <= 4096 with c in {9, 15, 25, 45, 75, 225}, 16 | L
// (3600 = 225 x 16 is Tab. 2's side); noise_len_supported() agrees. These lengths run CTAs
// whose thread count need not be a multiple of 32 (225 threads at 3600). They are compiled in
// a translation unit of their own (noise_extra.cu).
#define FR_NOISE_EXTRA_DISPATCH(len, F, ...)                          \
  switch (len) {                                                      \
    case 144: return F<144>(__VA_ARGS__);                             \
    case 288: return F<288>(__VA_ARGS__);                             \
    case 576: return F<576>(__VA_ARGS__);                             \
    case 1152: return F<1152>(__VA_ARGS__);                           \
    case 2304: return F<2304>(__VA_ARGS__);                           \
    case 240: return F<240>(__VA_ARGS__);                             \
    case 480: return F<480>(__VA_ARGS__);                             \
    case 960: return F<960>(__VA_ARGS__);                             \
    case 1920: return F<1920>(__VA_ARGS__);                           \
    case 3840: return F<3840>(__VA_ARGS__);                           \
    case 400: return F<400>(__VA_ARGS__);                             \
    case 800: return F<800>(__VA_ARGS__);                             \
    case 1600: return F<1600>(__VA_ARGS__);                           \
    case 3200: return F<3200>(__VA_ARGS__);                           \
    case 720: return F<720>(__VA_ARGS__);                             \
    case 1440: return F<1440>(__VA_ARGS__);                           \
    case 2880: return F<2880>(__VA_ARGS__);                           \
    case 1200: return F<1200>(__VA_ARGS__);                           \
    case 2400: return F<2400>(__VA_ARGS__);                           \
    case 3600: return F<3600>(__VA_ARGS__);                           \
    default:                                                          \
      ::fr::set_error("noise-pass length %d unsupported", (int)(len)); \
      return FR_EUNSUPPORTED;                                         \
  }

// Sum of one double per thread over the CTA into *dst (atomicAdd), for any blockDim.x (the
// last warp may be partial: its shuffles name only the lanes that exist, and values read from
// lanes past the end are discarded).
__device__ __forceinline__ void block_sum_atomic(double* dst, double acc) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  const int nl = min(32, (int)blockDim.x - 32 * wid);  // lanes in this warp
  const unsigned mask = nl == 32 ? 0xffffffffu : ((1u << nl) - 1u);
  for (int o = 16; o > 0; o >>= 1) {
    const double v = __shfl_down_sync(mask, acc, o);
    if (lane + o < nl) acc += v;
  }
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (wid == 0) {
    acc = lane < nw ? red[lane] : 0.0;
    const int nl0 = min(32, (int)blockDim.x);
    const unsigned mask0 = nl0 == 32 ? 0xffffffffu : ((1u << nl0) - 1u);
    for (int o = 16; o > 0; o >>= 1) {
      const double v = __shfl_down_sync(mask0, acc, o);
      if (lane + o < nl0) acc += v;
    }
    if (lane == 0) atomicAdd(dst, acc);
  }
}

}  // namespace fr
