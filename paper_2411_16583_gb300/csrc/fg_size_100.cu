// Pass kernels of transform length 100: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize100 {
  RegisterSize100() {
    register_size_ops_f(make_size_ops<float, 100>());
    register_size_ops_d(make_size_ops<double, 100>());
    register_size_ops_ff(make_size_ops_ff<100>());
  }
} register_size_100;
}  // namespace
}  // namespace fg
