// Pass kernels of transform length 96, both precisions.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize96 {
  RegisterSize96() {
    register_size_ops_f(make_size_ops<float, 96>());
    register_size_ops_d(make_size_ops<double, 96>());
  }
} register_size_96;
}  // namespace
}  // namespace fg
