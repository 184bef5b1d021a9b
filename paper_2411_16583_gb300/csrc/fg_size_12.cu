// Pass kernels of transform length 12: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize12 {
  RegisterSize12() {
    register_size_ops_f(make_size_ops<float, 12>());
    register_size_ops_d(make_size_ops<double, 12>());
    register_size_ops_ff(make_size_ops_ff<12>());
  }
} register_size_12;
}  // namespace
}  // namespace fg
