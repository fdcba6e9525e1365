"""The binding's constants against the C header they mirror: every enumerator
and #define of include/hydro.h that paper_2210_06437_gb300/hydro.py restates
(status codes, precisions, flux forms, parameter keys, the batch-id flag, the
limits) has the header's value, and every parameter key of the header has a
counterpart in the binding."""
import os
import re

from paper_2210_06437_gb300 import hydro as HY

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hydro.h")


def _header_values():
    text = open(HEADER).read()
    vals = {}
    for name, v in re.findall(r"\b(HYDRO_[A-Z0-9_]+)\s*=\s*(-?(?:0x[0-9a-fA-F]+|\d+))", text):
        vals[name] = int(v, 0)
    for name, v in re.findall(r"#define\s+(HYDRO_[A-Z0-9_]+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))", text):
        vals[name] = int(v, 0)
    return vals


def test_parameter_keys_match_the_header():
    vals = _header_values()
    keys = {k[len("HYDRO_PARAM_"):]: v for k, v in vals.items() if k.startswith("HYDRO_PARAM_")}
    assert keys, "no HYDRO_PARAM_ enumerators found"
    for name, v in keys.items():
        assert getattr(HY, "PARAM_" + name) == v, name


def test_status_precision_and_flux_codes_match_the_header():
    vals = _header_values()
    for code, name in HY.STATUS.items():
        assert vals[name] == code, name
    assert vals["HYDRO_FP64"] == HY.HYDRO_FP64 and vals["HYDRO_MIXED"] == HY.HYDRO_MIXED
    assert vals["HYDRO_FLUX_KNP"] == HY.HYDRO_FLUX_KNP and vals["HYDRO_FLUX_KT"] == HY.HYDRO_FLUX_KT


def test_flags_and_limits_match_the_header():
    vals = _header_values()
    assert vals["HYDRO_ITEM_FLUX_ONLY"] == HY.ITEM_FLUX_ONLY
    assert vals["HYDRO_TOTALS_NOALLOC_MAX_SUBGRIDS"] == HY.TOTALS_NOALLOC_MAX_SUBGRIDS
    assert vals["HYDRO_RK3_RUN_MAX_STEPS"] == HY.RK3_RUN_MAX_STEPS
