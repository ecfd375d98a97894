// Compile-time-plan product kernels, float instantiations (see tf_ct_kernels.cuh).
#include "tf_ct_kernels.cuh"

namespace tfk {
TF_DEFINE_OOB_READER(oob_read_ct_f32)
TF_CT_DEFINE_DISPATCH(float, TF_CT_MENU_COLS_F32)

namespace {
struct MenuEntry { int n; int np; int r[4]; };
template <int... R> constexpr int count_of() { return (int)sizeof...(R); }
#define TF_CT_MENU_ENTRY(N, ...) {N, count_of<__VA_ARGS__>(), {__VA_ARGS__}},
const MenuEntry kMenu[] = {TF_CT_MENU(TF_CT_MENU_ENTRY)};
#undef TF_CT_MENU_ENTRY
}  // namespace

unsigned ct_pipe_status(bool clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, ctk::g_pipe_status, sizeof(v)) != cudaSuccess) return 0;
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(ctk::g_pipe_status, &z, sizeof(z));
  }
  return v;
}

int ct_menu_count() { return (int)(sizeof(kMenu) / sizeof(kMenu[0])); }
int ct_menu_length(int i) { return kMenu[i].n; }
int ct_menu_radices(int i, int* radices) {
  for (int p = 0; p < kMenu[i].np; ++p) radices[p] = kMenu[i].r[p];
  return kMenu[i].np;
}

namespace {
#define TF_CT_MENU_ENTRY(N, ...) {N, count_of<__VA_ARGS__>(), {__VA_ARGS__}},
const MenuEntry kMenuCols[] = {TF_CT_MENU_COLS_F32(TF_CT_MENU_ENTRY)};
#undef TF_CT_MENU_ENTRY
}  // namespace

int ct_menu_cols_radices(int n, int* radices) {  // single-precision column plans
  for (const MenuEntry& e : kMenuCols)
    if (e.n == n) {
      for (int p = 0; p < e.np; ++p) radices[p] = e.r[p];
      return e.np;
    }
  return 0;
}
}  // namespace tfk
