// Pass kernels of transform length 24: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize24 {
  RegisterSize24() {
    register_size_ops_f(make_size_ops<float, 24>());
    register_size_ops_d(make_size_ops<double, 24>());
    register_size_ops_ff(make_size_ops_ff<24>());
  }
} register_size_24;
}  // namespace
}  // namespace fg
