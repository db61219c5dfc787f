// rect_i32.cu — rectangular executor instantiated for int32 (modulo 2^32) sum / max / min.
#include "rect_launch.cuh"

namespace hp {
hp_status launch_rect_i32_sum(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpI32Sum>(np, cfg, a);
}
hp_status launch_rect_i32_max(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpI32Max>(np, cfg, a);
}
hp_status launch_rect_i32_min(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpI32Min>(np, cfg, a);
}
}  // namespace hp
