// Pass kernels of transform length 64: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize64 {
  RegisterSize64() {
    register_size_ops_f(make_size_ops<float, 64>());
    register_size_ops_d(make_size_ops<double, 64>());
    register_size_ops_ff(make_size_ops_ff<64>());
  }
} register_size_64;
}  // namespace
}  // namespace fg
