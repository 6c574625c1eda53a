// Register-kernel instances for class codes 399..454, code = ((la*7 + lb)*7 + lc)*7 + ld
// (see reg_kernel.cuh; split over several files so that they compile in parallel).
#include "reg_kernel.cuh"

namespace mdx {

cudaError_t launch_reg_part06(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled) {
  *handled = false;
  if (code < 399 || code >= 455) return cudaSuccess;
  const reg::RegLaunchFn f = reg::reg_pick<399>(code, std::make_integer_sequence<int, 56>{});
  if (!f) return cudaSuccess;
  *handled = true;
  return f(a, s);
}

}  // namespace mdx
