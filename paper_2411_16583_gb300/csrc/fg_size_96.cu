// Pass kernels of transform length 96: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize96 {
  RegisterSize96() {
    register_size_ops_f(make_size_ops<float, 96>());
    register_size_ops_d(make_size_ops<double, 96>());
    register_size_ops_ff(make_size_ops_ff<96>());
  }
} register_size_96;
}  // namespace
}  // namespace fg
