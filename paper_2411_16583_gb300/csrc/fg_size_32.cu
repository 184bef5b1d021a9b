// Pass kernels of transform length 32: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize32 {
  RegisterSize32() {
    register_size_ops_f(make_size_ops<float, 32>());
    register_size_ops_d(make_size_ops<double, 32>());
    register_size_ops_ff(make_size_ops_ff<32>());
  }
} register_size_32;
}  // namespace
}  // namespace fg
