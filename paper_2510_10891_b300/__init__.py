"""B300 (sm_103a) library for the LP relaxations of the successive-fixing
SCUC method: restarted HPR solve (Sec. 3), logic-driven fixing (Sec. 4.1)
and bound-propagation presolve (Sec. 4.2), behind the C ABI of
include/scuc_lp.h.  This package only marshals arguments to that library;
importing it does not load the library until it is first used."""
from .filtering import transmission_filter  # noqa: F401
from .lp import LP, default_params, fma_peak, info_dict, solve_batch  # noqa: F401
