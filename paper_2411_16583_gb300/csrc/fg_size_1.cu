// Pass kernels of transform length 1, both precisions.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize1 {
  RegisterSize1() {
    register_size_ops_f(make_size_ops<float, 1>());
    register_size_ops_d(make_size_ops<double, 1>());
  }
} register_size_1;
}  // namespace
}  // namespace fg
