// Pass kernels of transform length 48: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize48 {
  RegisterSize48() {
    register_size_ops_f(make_size_ops<float, 48>());
    register_size_ops_d(make_size_ops<double, 48>());
    register_size_ops_ff(make_size_ops_ff<48>());
  }
} register_size_48;
}  // namespace
}  // namespace fg
