// Pass kernels of transform length 16: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize16 {
  RegisterSize16() {
    register_size_ops_f(make_size_ops<float, 16>());
    register_size_ops_d(make_size_ops<double, 16>());
    register_size_ops_ff(make_size_ops_ff<16>());
  }
} register_size_16;
}  // namespace
}  // namespace fg
