// Pass kernels of transform length 1: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize1 {
  RegisterSize1() {
    register_size_ops_f(make_size_ops<float, 1>());
    register_size_ops_d(make_size_ops<double, 1>());
    register_size_ops_ff(make_size_ops_ff<1>());
  }
} register_size_1;
}  // namespace
}  // namespace fg
