// Pass kernels of transform length 512: FP32, FP64 and the float-float residual passes.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize512 {
  RegisterSize512() {
    register_size_ops_f(make_size_ops<float, 512>());
    register_size_ops_d(make_size_ops<double, 512>());
    register_size_ops_ff(make_size_ops_ff<512>());
  }
} register_size_512;
}  // namespace
}  // namespace fg
