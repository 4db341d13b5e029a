// Sum of partial results (Thm 4.2): the weighted count of a formula is the
// sum, over the assignments eta of the sliced variables, of the counts of
// the formula conditioned on eta.  Index slicing across processes (Alg. 3
// with one share of the slice assignments per process) leaves one partial
// sum per process; this adds them.  Host only.
#include <cmath>
#include <cstring>

#include "internal.h"

using namespace wmc;

extern "C" int wmc_combine_results(const wmc_result *parts, int64_t n, wmc_result *out) {
  if (!out || n < 0 || (n > 0 && !parts)) { set_error("bad argument"); return WMC_EINVAL; }
  // the largest binary exponent of the nonzero parts (value = fr * 2^e,
  // fr in [0.5, 1)); every part is brought to that exponent, so the sum
  // stays in [-n, n] whatever the parts' own exponents are
  bool any = false;
  int64_t emax = 0;
  uint32_t flags_or = 0;
  bool all_exact = n > 0;
  double bound = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const wmc_result &r = parts[i];
    if (!std::isfinite(r.mant)) { set_error("part %lld is not finite", (long long)i); return WMC_EINVAL; }
    flags_or |= r.flags;
    all_exact = all_exact && (r.flags & WMC_FLAG_EXACT_INT);
    bound = std::fmax(bound, r.rel_err_bound);
    if (r.mant == 0.0) continue;
    int fe = 0;
    std::frexp(r.mant, &fe);
    const int64_t e = r.exp2 + fe;
    if (!any || e > emax) emax = e;
    any = true;
  }
  // parts in order, each scaled by 2^(its exponent - emax): exact unless it
  // falls below the float64 range, which is below the sum's last bit
  double sum = 0.0;
  if (any)
    for (int64_t i = 0; i < n; ++i) {
      const wmc_result &r = parts[i];
      if (r.mant == 0.0) continue;
      int fe = 0;
      const double fr = std::frexp(r.mant, &fe);
      const int64_t d = r.exp2 + fe - emax;  // <= 0
      sum += d < -1100 ? 0.0 : std::ldexp(fr, (int)d);
    }
  std::memset(out, 0, sizeof(*out));
  int fe = 0;
  const double fr = std::frexp(sum, &fe);
  out->mant = fr;
  out->exp2 = sum == 0.0 ? 0 : emax + fe;
  out->log10 = sum == 0.0 ? -INFINITY : std::log10(std::fabs(fr)) + (double)out->exp2 * std::log10(2.0);
  // exact integer sums stay exact while the total is below 2^53; other
  // flags are kept if any part carries them
  out->flags = flags_or & ~WMC_FLAG_EXACT_INT;
  if (all_exact && sum != 0.0 && out->exp2 <= 53) out->flags |= WMC_FLAG_EXACT_INT;
  if (all_exact && sum == 0.0) out->flags |= WMC_FLAG_EXACT_INT;
  // nonnegative parts: the largest part bound plus one float64 rounding
  // per addition
  out->rel_err_bound = bound + (double)(n > 1 ? n - 1 : 0) * std::ldexp(1.0, -53);
  return WMC_OK;
}
