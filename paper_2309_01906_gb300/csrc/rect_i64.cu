// rect_i64.cu — rectangular executor instantiated for int64 sum / max / min of int32 inputs.
#include "rect_launch.cuh"

namespace hp {
hp_status launch_rect_i64_sum(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpI64Sum>(np, cfg, a);
}
hp_status launch_rect_i64_max(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpI64Max>(np, cfg, a);
}
hp_status launch_rect_i64_min(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpI64Min>(np, cfg, a);
}
}  // namespace hp
