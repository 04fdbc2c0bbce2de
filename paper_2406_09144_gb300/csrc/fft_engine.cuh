// Shared-memory FFT engine and the generic row / column pass kernels.
//
// A CTA holds B sequences of length L = 2^LOG2L in shared memory (sequence b at b * LP,
// element i at spad(i)), 16 complex points per thread, and runs the Stockham stages of
// fft_core.cuh with register-held butterflies. Row passes read rows that are contiguous in
// global memory; column passes read B adjacent columns (coalesced across the B columns of each
// row) and transpose them into the same shared layout.
#pragma once
#include "fr_internal.cuh"

namespace fr {

template <int LOG2L>
struct FftCfg {
  static constexpr int L = 1 << LOG2L;
  static constexpr int B = (L >= 4096) ? 1 : 4096 / L;   // sequences per CTA
  static constexpr int NT = (B * L) / 16;                 // threads: 16 points each
  static constexpr int LP = spad_len(L) + 1;              // odd stride between sequences
  static constexpr size_t SMEM = size_t(B) * LP * sizeof(float2);
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
      for (int r = 0; r < R; ++r) {
        float2 x = src[spad(j + r * LR)];
        if constexpr (ST > 0) {
          if (r > 0) {
            float2 w = __ldg(&tw[r * k * TSTEP]);
            if (DIR > 0) w.y = -w.y;
            x = cmul(x, w);
          }
        }
        v[q][r] = x;
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

// Row pass: sequences are rows. Op provides
//   float2 load(int seq, int i)                      for i in [0, L)
//   int nout() const; double store(int seq, int o, SeqView v)   for o in [0, nout)
//   int nseq() const; void finish(int seq0, double acc)  (per-thread sum of store results)
template <int LOG2L, int DIR, class Op>
__global__ void __launch_bounds__(FftCfg<LOG2L>::NT) fft_rows_kernel(Op op,
                                                                      const float2* __restrict__ tw) {
  using C = FftCfg<LOG2L>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  extern __shared__ float2 smem[];
  const int nseq = op.nseq();
  const int seq0 = blockIdx.x * B;
  for (int idx = threadIdx.x; idx < B * L; idx += NT) {
    const int b = idx / L, i = idx % L;
    const int sq = seq0 + b;
    smem[b * LP + spad(i)] = (sq < nseq) ? op.load(sq, i) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_stages<LOG2L, 0, DIR>(smem, tw);
  const int nout = op.nout();
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < B * nout; idx += NT) {
    const int b = idx / nout, o = idx % nout;
    const int sq = seq0 + b;
    if (sq < nseq) acc += op.store(sq, o, SeqView{smem + b * LP});
  }
  op.finish(seq0, acc);
}

// Column pass: sequences are columns; blockIdx.y selects an image for ops that batch images.
// Op provides
//   float2 load(int i, int col)   i in [0, L)
//   void after_load(int col0)     (e.g. zero the source once every CTA thread has loaded)
//   void mid(float2* s, int col0) (between the two transforms when TWO is set)
//   int nout() const; void store(int o, int col, SeqView v)
//   int ncol() const
template <int LOG2L, int DIR, int DIR2, bool TWO, class Op>
__global__ void __launch_bounds__(FftCfg<LOG2L>::NT) fft_cols_kernel(Op op,
                                                                      const float2* __restrict__ tw) {
  using C = FftCfg<LOG2L>;
  constexpr int L = C::L, B = C::B, NT = C::NT, LP = C::LP;
  extern __shared__ float2 smem[];
  const int ncol = op.ncol();
  const int col0 = blockIdx.x * B;
  for (int idx = threadIdx.x; idx < B * L; idx += NT) {
    const int i = idx / B, c = idx % B;
    const int col = col0 + c;
    smem[c * LP + spad(i)] = (col < ncol) ? op.load(i, col) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  op.after_load(col0);
  fft_stages<LOG2L, 0, DIR>(smem, tw);
  if constexpr (TWO) {
    op.mid(smem, col0);
    __syncthreads();
    fft_stages<LOG2L, 0, DIR2>(smem, tw);
  }
  const int nout = op.nout();
  for (int idx = threadIdx.x; idx < B * nout; idx += NT) {
    const int o = idx / B, c = idx % B;
    const int col = col0 + c;
    if (col < ncol) op.store(o, col, SeqView{smem + c * LP});
  }
}

// The column kernel calls op.after_load(col0) and op.mid(smem, col0); ops implement them as
// templates on the CTA shape, which this wrapper fixes.
template <int LOG2L, class Op>
struct ColOp : Op {
  using C = FftCfg<LOG2L>;
  __device__ void after_load(int col0) const { Op::template after_load<C::B, C::NT, C::L>(col0); }
  __device__ void mid(float2* s, int col0) const {
    Op::template mid<C::B, C::NT, C::L, C::LP>(s, col0);
  }
};

template <int LOG2L, int DIR, class Op>
int launch_rows(const Op& op, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LOG2L>;
  const int nblk = (op.nseq() + C::B - 1) / C::B;
  if (nblk == 0) return FR_OK;
  auto kern = fft_rows_kernel<LOG2L, DIR, Op>;
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    attr = true;
  }
  kern<<<nblk, C::NT, C::SMEM, s>>>(op, tw);
  FR_LAUNCHED();
  return FR_OK;
}

template <int LOG2L, int DIR, int DIR2, bool TWO, class Op>
int launch_cols(const Op& op, int nimg, const float2* tw, cudaStream_t s) {
  using C = FftCfg<LOG2L>;
  const int nblk = (op.ncol() + C::B - 1) / C::B;
  if (nblk == 0 || nimg == 0) return FR_OK;
  auto kern = fft_cols_kernel<LOG2L, DIR, DIR2, TWO, Op>;
  static bool attr = false;
  if (!attr) {
    FR_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    attr = true;
  }
  kern<<<dim3(nblk, nimg), C::NT, C::SMEM, s>>>(op, tw);
  FR_LAUNCHED();
  return FR_OK;
}

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
