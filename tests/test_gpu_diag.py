"""The phase-boundary diagnostic runs on the device and reports finite positive times for
both forms (a kernel per phase in a graph with programmatic dependent launch, and a grid
barrier in one cooperative kernel) without its bounded barrier wait giving up."""
import math

import pytest

from paper_2503_15078_b300 import measure_phase_boundaries

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ctas_per_sm", [1, 2])
def test_phase_boundary_measurement(ctas_per_sm):
    g_us, b_us = measure_phase_boundaries(n_phases=64, ctas_per_sm=ctas_per_sm)
    print(f"\n{ctas_per_sm} CTA/SM: graph with PDL {g_us:.3f} us, grid barrier {b_us:.3f} us "
          "per boundary")
    assert math.isfinite(g_us) and math.isfinite(b_us)
    assert 0.0 < g_us < 1e3 and 0.0 < b_us < 1e3
