"""The binding checks array dtypes before calling the library (no GPU needed):
a float64 or float16 array passed where the C ABI reads float32 would be
reinterpreted and give silently wrong results, so it raises ValueError."""
import os

import pytest

import paper_2411_03289_gb300 as gp


@pytest.mark.skipif(not os.path.exists(gp.LIB_PATH), reason="library not built")
@pytest.mark.parametrize("bad", ["costs", "u_tilde", "U_nom", "U_new", "weights"])
def test_noalloc_refuses_non_float32(bad):
    import torch
    K, T = 8, 3
    arrs = dict(costs=torch.zeros(K), u_tilde=torch.zeros(T, K, 2), U_nom=torch.zeros(T, 2),
                U_new=torch.zeros(T, 2), weights=torch.zeros(K))
    arrs[bad] = arrs[bad].double()
    with pytest.raises(ValueError, match="dtype"):
        gp.mppi_update_noalloc(arrs["costs"], arrs["u_tilde"], arrs["U_nom"], arrs["U_new"],
                               arrs["weights"], K, T, 1.0)
