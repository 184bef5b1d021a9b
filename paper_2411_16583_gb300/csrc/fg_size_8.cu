// Pass kernels of transform length 8: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize8 {
  RegisterSize8() {
    register_size_ops_f(make_size_ops<float, 8>());
    register_size_ops_d(make_size_ops<double, 8>());
    register_size_ops_ff(make_size_ops_ff<8>());
  }
} register_size_8;
}  // namespace
}  // namespace fg
