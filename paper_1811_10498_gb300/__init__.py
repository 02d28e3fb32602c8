"""GB300-native PFAC DNA match scan (arXiv 1811.10498).

The scan runs in the CUDA library ``libpfac.so`` (C ABI in ``include/pfac.h``); this
package is its thin Python binding plus the launch autotuner, the batched-read driver,
the serving loop and the overlapped scanner for texts in host memory. ``datagen`` makes
the seeded synthetic inputs.
"""
from ._binding import (  # noqa: F401
    CODE, STATUS, PfacError, Table, lib, pack, pfac_build, pfac_build_file, pfac_debug_timeout_probe, pfac_destroy,
    pfac_device_status, pfac_export, pfac_export_shortcuts, pfac_get_config, pfac_info, pfac_info_ex, pfac_match,
    pfac_match_all, pfac_match_batched, pfac_match_compact, pfac_match_packed, pfac_match_packed_noalloc, pfac_pack,
    pfac_set_config, read_text_file,
)
