// Pass kernels of transform length 80: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize80 {
  RegisterSize80() {
    register_size_ops_f(make_size_ops<float, 80>());
    register_size_ops_d(make_size_ops<double, 80>());
    register_size_ops_ff(make_size_ops_ff<80>());
  }
} register_size_80;
}  // namespace
}  // namespace fg
