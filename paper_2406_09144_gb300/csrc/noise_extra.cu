// Noise passes (Sec. 3.3.3) at the image sides whose odd part has several factors 3 and 5
// (c 2^k <= 4096, 16 | L, c in {9, 15, 25, 45, 75, 225}; Tab. 2's 3600 = 225 x 16), compiled
// apart from noise.cu so that the two compile in parallel.
#include "noise_ops.cuh"

namespace fr {

bool noise_extra_len(int L) {
  if (L < 144 || L > 4096 || L % 16 != 0) return false;
  const int c = odd_part(L);
  return c == 9 || c == 15 || c == 25 || c == 45 || c == 75 || c == 225;
}

int nk1_extra(int len, const NK1Op& op, int n, const float2* tw, cudaStream_t s) { FR_NOISE_EXTRA_DISPATCH(len, run_nk1, op, n, tw, s); }
int nk2_extra(int len, const NK2Op& op, int n, const float2* tw, cudaStream_t s) { FR_NOISE_EXTRA_DISPATCH(len, run_nk2, op, n, tw, s); }
int nk3_extra(int len, const NK3Op& op, int n, const float2* tw, cudaStream_t s) { FR_NOISE_EXTRA_DISPATCH(len, run_nk3, op, n, tw, s); }
int nkf_extra(int len, const NKFOp& op, int n, const float2* tw, cudaStream_t s) { FR_NOISE_EXTRA_DISPATCH(len, run_nkf, op, n, tw, s); }

}  // namespace fr
