// Pass kernels of transform length 128: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize128 {
  RegisterSize128() {
    register_size_ops_f(make_size_ops<float, 128>());
    register_size_ops_d(make_size_ops<double, 128>());
    register_size_ops_ff(make_size_ops_ff<128>());
  }
} register_size_128;
}  // namespace
}  // namespace fg
