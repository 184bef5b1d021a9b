// Pass kernels of transform length 80, both precisions.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize80 {
  RegisterSize80() {
    register_size_ops_f(make_size_ops<float, 80>());
    register_size_ops_d(make_size_ops<double, 80>());
  }
} register_size_80;
}  // namespace
}  // namespace fg
