// placeholder, replaced by the tcgen05 emulation below
#include "emu.h"
bool emu_wanted(Ctx& c, const GemmPlan& g, const std::string& site) { return false; }
EmuPlan* emu_plan(Ctx&, const GemmPlan&, const Tensor*, const Tensor*, bool, bool) { return nullptr; }
void emu_run(Ctx&, EmuPlan*, const GemmPlan&, const cplx*, const cplx*, cplx*, int64_t, int64_t, int64_t, cplx, bool) {}
void emu_release(Ctx&) {}
