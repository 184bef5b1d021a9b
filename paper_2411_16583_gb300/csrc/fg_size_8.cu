// Pass kernels of transform length 8, both precisions.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize8 {
  RegisterSize8() {
    register_size_ops_f(make_size_ops<float, 8>());
    register_size_ops_d(make_size_ops<double, 8>());
  }
} register_size_8;
}  // namespace
}  // namespace fg
