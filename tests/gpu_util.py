"""Helpers for the GPU tests: the CUDA path through the C ABI, the oracle
beside it, and the comparison rules."""
import numpy as np

import oracle
from paper_2208_12964_gb300 import synth

ORACLE_KEYS = dict(oracle.Problem._fields_)


def oracle_for(spec, threads=8, weight_mode=None, store_form=None):
    d = {k: v for k, v in spec.items() if k in ORACLE_KEYS}
    d["weight_mode"] = spec.get("weight_mode", oracle.LENGTH) if weight_mode is None else weight_mode
    d["store_form"] = spec.get("store_form", oracle.STORE_ROWS) if store_form is None else store_form
    if spec.get("custom_sectors") is not None:
        d["custom_sectors"] = spec["custom_sectors"]
    return oracle.Oracle(d, threads=threads)


class Gpu:
    """One libuspg context for a workload description."""

    def __init__(self, spec, dtype=None, weight_mode=None, store_form=None):
        from paper_2208_12964_gb300 import uspg

        self.U = uspg
        dtype = uspg.F32 if dtype is None else dtype
        g, s, o, self._keep = uspg.descs_from_spec(spec, dtype, weight_mode, store_form)
        self.ctx = uspg.uspg_create(g, s, o)
        self.spec = spec

    def build(self):
        self.U.uspg_build_coeffs(self.ctx)
        return self

    def stats(self):
        return self.U.uspg_coeff_stats(self.ctx)

    def row(self, view, ray):
        c, w = self.U.uspg_get_row(self.ctx, view, ray)
        o = np.argsort(c, kind="stable")
        return c[o], w[o]

    def close(self):
        if self.ctx:
            self.U.uspg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def assert_rows_equal(gcells, gw, ocells, ow, wtol=1e-6, where=""):
    assert np.array_equal(gcells, ocells), f"cell lists differ {where}: gpu {gcells[:8]}.. oracle {ocells[:8]}.."
    if len(ow):
        rel = np.abs(gw - ow) / np.abs(ow)
        assert rel.max() <= wtol, f"weights differ {where}: max rel {rel.max():.3e}"


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
