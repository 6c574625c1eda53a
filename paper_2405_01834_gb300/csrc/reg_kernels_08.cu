// Register-kernel instances for class codes 539..699, code = ((la*7 + lb)*7 + lc)*7 + ld
// (see reg_kernel.cuh; split over several files so that they compile in parallel).
#include "reg_kernel.cuh"

namespace mdx {

cudaError_t launch_reg_part08(int code, const QuartetLaunch& a, cudaStream_t s, bool* handled) {
  *handled = false;
  if (code < 539 || code >= 700) return cudaSuccess;
  const reg::RegLaunchFn f = reg::reg_pick<539>(code, std::make_integer_sequence<int, 161>{});
  if (!f) return cudaSuccess;
  *handled = true;
  return f(a, s);
}

}  // namespace mdx
