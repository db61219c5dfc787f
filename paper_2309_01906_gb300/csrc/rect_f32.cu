// rect_f32.cu — rectangular executor instantiated for FP32 sums (plain and compensated).
#include "rect_launch.cuh"

namespace hp {
hp_status launch_rect_f32_sum(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpF32Sum>(np, cfg, a);
}
hp_status launch_rect_f32_comp(const NestPlan& np, LaunchCfg& cfg, const RectArgs& a) {
  return launch_rect<OpF32Comp>(np, cfg, a);
}
}  // namespace hp
