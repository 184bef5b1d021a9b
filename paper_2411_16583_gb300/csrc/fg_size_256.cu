// Pass kernels of transform length 256, both precisions.
#include "fg_launch.cuh"

namespace fg {
namespace {
struct RegisterSize256 {
  RegisterSize256() {
    register_size_ops_f(make_size_ops<float, 256>());
    register_size_ops_d(make_size_ops<double, 256>());
  }
} register_size_256;
}  // namespace
}  // namespace fg
