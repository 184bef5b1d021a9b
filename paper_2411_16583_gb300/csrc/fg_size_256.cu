// Pass kernels of transform length 256: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize256 {
  RegisterSize256() {
    register_size_ops_f(make_size_ops<float, 256>());
    register_size_ops_d(make_size_ops<double, 256>());
    register_size_ops_ff(make_size_ops_ff<256>());
  }
} register_size_256;
}  // namespace
}  // namespace fg
