// Shared-memory FFT engine and the generic FFT pass kernel.
//
// Every pass reads the sequences it transforms from contiguous memory: a CTA loads B
// sequences of length L = 2^LOG2L (register-staged, 16 complex values per thread, all loads in
// flight before the first shared-memory store), runs the Stockham stages of fft_core.cuh
// on them in shared memory (sequence b at b * LP, element i at spad(i)), and hands them to the
// pass's store, which writes either along the sequence (row-major) or across the B sequences
// (transposed: consecutive threads write consecutive sequences of one output index). The
// transposed store is how a pass produces the layout the next pass reads contiguously, so no
// pass ever reads a column.
#pragma once
#include "fr_internal.cuh"

namespace fr {

template <int LOG2L>
struct FftCfg {
  static constexpr int L = 1 << LOG2L;
  // L = 8192 and 16384 run one sequence per CTA so that two CTAs share an SM and overlap
  // their load, transform and store phases; L = 4096 keeps two (16-byte transposed stores)
  static constexpr int B = (L >= 8192) ? 1 : (L >= 4096 ? 2 : 4096 / L);
  static constexpr int NT = (B * L) / 16;     // threads: 16 points each
  static constexpr int LP = spad_len(L) + 1;  // odd stride between sequences
  static constexpr size_t SMEM = size_t(B) * LP * sizeof(float2);
  // CTAs per SM the register budget is sized for: four at L = 2048 (64 registers, no spills)
  static constexpr int MINB = NT >= 1024 ? 1 : (NT >= 512 || LOG2L < 11 ? 2 : 4);
  static constexpr int MINB_SUM = NT >= 512 ? 1 : 2;  // summing and multi-output passes
  static constexpr int MINB_TWO = NT >= 1024 ? 1 : 2;  // two-transform passes
};

constexpr int ns_before(int log2l, int st) {
  int b = 0;
  for (int s = 0; s < st; ++s) b += stage_bits(log2l, s);
  return 1 << b;
}

template <int LOG2L, int ST, int DIR>
__device__ __forceinline__ void fft_stages(float2* s, const float2* __restrict__ tw) {
  if constexpr (ST < num_stages(LOG2L)) {
    using C = FftCfg<LOG2L>;
    constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
    constexpr int R = 1 << stage_bits(LOG2L, ST);
    constexpr int NS = ns_before(LOG2L, ST);
    constexpr int LR = L / R;
    constexpr int NTASK = B * LR;
    static_assert(NTASK % NT == 0, "tasks must divide evenly among threads");
    constexpr int TPT = NTASK / NT;
    constexpr int TSTEP = L / (NS * R);
    float2 v[TPT][R];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int t = threadIdx.x + q * NT;
      const int b = t / LR, j = t % LR;
      const int k = j & (NS - 1);
      const float2* src = s + b * LP;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = src[spad(j + r * LR)];
      if constexpr (ST > 0) {
        // w^r for r < R from the table entries w^1, w^2, w^4, w^8 (w = exp(dir 2 pi i k / (NS R)))
        // and at most two further products per factor: a few ulp, log2(R) loads per butterfly
        constexpr int LB = stage_bits(LOG2L, ST);
        float2 pw[LB];
#pragma unroll
        for (int e = 0; e < LB; ++e) {
          float2 w = __ldg(&tw[(k * TSTEP) << e]);
          if (DIR > 0) w.y = -w.y;
          pw[e] = w;
        }
        float2 wr[R];
        twiddle_rec<R, 1>(v[q], pw, wr);
      }
      dft_r<R, DIR>(v[q]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int t = threadIdx.x + q * NT;
      const int b = t / LR, j = t % LR;
      const int k = j & (NS - 1);
      float2* dst = s + b * LP;
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[spad(base + r * NS)] = v[q][r];
    }
    __syncthreads();
    fft_stages<LOG2L, ST + 1, DIR>(s, tw);
  }
}

// Read-only view of one sequence in shared memory.
struct SeqView {
  const float2* p;
  __device__ __forceinline__ float2 operator[](int i) const { return p[spad(i)]; }
};

// Generic pass. blockIdx.x selects B consecutive sequences, blockIdx.y an image (ops that batch
// images use it). Op provides:
//   static constexpr bool TRANSPOSED   store mapping (see above)
//   static constexpr bool TWO          second transform (DIR2) after mid()
//   int nseq() const, int nout() const      (host and device)
//   float2 load(int seq, int i)        element i of the sequence (zero padding costs no load)
//   void after_load(int seq0, int nb)  after every thread's loads have landed
//   void mid(float2* s, int seq0)      between the transforms (TWO)
//   double store(int seq, int o, SeqView v)   o < nout(); per-thread results are summed
//   void finish(int seq0, double acc)
template <int LOG2L, int DIR, int DIR2, class Op>
__global__ void __launch_bounds__(FftCfg<LOG2L>::NT,
                                  Op::TWO ? FftCfg<LOG2L>::MINB_TWO : FftCfg<LOG2L>::MINB)
    fft_pass_kernel(Op op, const float2* __restrict__ tw) {
  using C = FftCfg<LOG2L>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  constexpr int PER = B * L / NT;
  extern __shared__ float2 smem[];
  const int nseq = op.nseq();
  const int seq0 = blockIdx.x * B;
  float2 r[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * NT;
    const int b = idx / L, i = idx % L;
    r[k] = (seq0 + b < nseq) ? op.load(seq0 + b, i) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * NT;
    smem[(idx / L) * LP + spad(idx % L)] = r[k];
  }
  __syncthreads();
  op.after_load(seq0, min(B, nseq - seq0));
  fft_stages<LOG2L, 0, DIR>(smem, tw);
  if constexpr (Op::TWO) {
    op.template mid<B, NT, L, LP>(smem, seq0);
    __syncthreads();
    fft_stages<LOG2L, 0, DIR2>(smem, tw);
  }
  const int nout = op.nout();
  double acc = 0.0;
  if constexpr (Op::TRANSPOSED) {
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

template <int LOG2L, int DIR, int DIR2, class Op>
int launch_pass(const Op& op, int nimg, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LOG2L>;
  const int nblk = (op.nseq() + C::B - 1) / C::B;
  if (nblk == 0 || nimg == 0) return FR_OK;
  auto kern = fft_pass_kernel<LOG2L, DIR, DIR2, Op>;
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    attr = true;
  }
  kern<<<dim3(nblk, nimg), C::NT, C::SMEM, s>>>(op, tw);
  FR_LAUNCHED();
  return FR_OK;
}

// Summing pass: for each of op.nterms() inputs per sequence (blockIdx.x selects B sequences),
// load, transform and add op.value(t, seq, o, view) into per-thread accumulators kept in shared
// memory after the transform buffer; one op.store(seq, o, sum) per output at the end. The next
// input's loads are issued before the current one is transformed. Row-major outputs (o fastest),
// nout <= L.
//   float2 load(int t, int seq, int i); float value(int t, int seq, int o, SeqView v);
//   void store(int seq, int o, float sum)
template <int LOG2L, int DIR, class Op>
__global__ void __launch_bounds__(FftCfg<LOG2L>::NT, FftCfg<LOG2L>::MINB_SUM)
    fft_pass_sum_kernel(Op op, const float2* __restrict__ tw) {
  using C = FftCfg<LOG2L>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  constexpr int PER = B * L / NT;
  extern __shared__ float2 smem[];
  float* accs = reinterpret_cast<float*>(smem + B * LP);  // [B * nout], one entry per output
  const int nseq = op.nseq(), nout = op.nout(), nterm = op.nterms();
  const int seq0 = blockIdx.x * B;
#pragma unroll
  for (int k = 0; k < PER; ++k) accs[threadIdx.x + k * NT] = 0.f;  // B * nout <= B * L
  float2 r[PER];
  auto fetch = [&](int t) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + k * NT;
      const int b = idx / L, i = idx % L;
      r[k] = (seq0 + b < nseq) ? op.load(t, seq0 + b, i) : make_float2(0.f, 0.f);
    }
  };
  if (nterm > 0) fetch(0);
  for (int t = 0; t < nterm; ++t) {
    if (t > 0) __syncthreads();  // the previous term's outputs have been read
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + k * NT;
      smem[(idx / L) * LP + spad(idx % L)] = r[k];
    }
    __syncthreads();
    if (t + 1 < nterm) fetch(t + 1);
    fft_stages<LOG2L, 0, DIR>(smem, tw);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + k * NT;
      if (idx < B * nout) {
        const int b = idx / nout, o = idx % nout;
        if (seq0 + b < nseq) accs[idx] += op.value(t, seq0 + b, o, SeqView{smem + b * LP});
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * NT;
    if (idx < B * nout) {
      const int b = idx / nout, o = idx % nout;
      if (seq0 + b < nseq) op.store(seq0 + b, o, accs[idx]);
    }
  }
}

template <int LOG2L, int DIR, class Op>
int launch_pass_sum(const Op& op, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LOG2L>;
  const int nblk = (op.nseq() + C::B - 1) / C::B;
  if (nblk == 0) return FR_OK;
  auto kern = fft_pass_sum_kernel<LOG2L, DIR, Op>;
  constexpr size_t smem = C::SMEM + size_t(C::B) * C::L * sizeof(float);
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
template <int LOG2L, int DIR, class Op>
__global__ void __launch_bounds__(FftCfg<LOG2L>::NT, FftCfg<LOG2L>::MINB_SUM)
    fft_pass_multi_kernel(Op op, const float2* __restrict__ tw) {
  using C = FftCfg<LOG2L>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  constexpr int PER = B * L / NT;
  extern __shared__ float2 smem[];
  const int nseq = op.nseq(), nout = op.nout(), nterm = op.nterms();
  const int seq0 = blockIdx.x * B;
  float2 r[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * NT;
    const int b = idx / L, i = idx % L;
    r[k] = (seq0 + b < nseq) ? op.load(seq0 + b, i) : make_float2(0.f, 0.f);
  }
  for (int t = 0; t < nterm; ++t) {
    if (t > 0) __syncthreads();  // the previous transform's outputs have been read
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = threadIdx.x + k * NT;
      smem[(idx / L) * LP + spad(idx % L)] = op.prep(t, r[k]);
    }
    __syncthreads();
    fft_stages<LOG2L, 0, DIR>(smem, tw);
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

template <int LOG2L, int DIR, class Op>
int launch_pass_multi(const Op& op, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LOG2L>;
  const int nblk = (op.nseq() + C::B - 1) / C::B;
  if (nblk == 0) return FR_OK;
  auto kern = fft_pass_multi_kernel<LOG2L, DIR, Op>;
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

// Defaults for the optional parts of an op.
struct OpBase {
  static constexpr bool TRANSPOSED = false;
  static constexpr bool TWO = false;
  __device__ void after_load(int, int) const {}
  template <int B, int NT, int L, int LP>
  __device__ void mid(float2*, int) const {}
  __device__ void finish(int, double) const {}
};

// Dispatch a templated functor on a runtime log2 length in [5, 14].
#define FR_LOG2_DISPATCH(log2l, F, ...)                      \
  switch (log2l) {                                           \
    case 5: return F<5>(__VA_ARGS__);                        \
    case 6: return F<6>(__VA_ARGS__);                        \
    case 7: return F<7>(__VA_ARGS__);                        \
    case 8: return F<8>(__VA_ARGS__);                        \
    case 9: return F<9>(__VA_ARGS__);                        \
    case 10: return F<10>(__VA_ARGS__);                      \
    case 11: return F<11>(__VA_ARGS__);                      \
    case 12: return F<12>(__VA_ARGS__);                      \
    case 13: return F<13>(__VA_ARGS__);                      \
    case 14: return F<14>(__VA_ARGS__);                      \
    default:                                                 \
      ::fr::set_error("FFT length 2^%d unsupported", log2l); \
      return FR_EUNSUPPORTED;                                \
  }

}  // namespace fr
