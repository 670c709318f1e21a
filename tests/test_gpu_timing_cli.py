"""The stencil timing command line (paper_2309_10292_gb300.timing)."""
import json

import pytest

from tests.gpu_util import need_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("argv,kernel", [
    (["--L", "16", "--steps", "3", "--plan", "zmarch,16,4,8"], 2),
    (["--L", "16", "--dtype", "f64", "--arith", "ds", "--steps", "2", "--plan", "naive"], 1),
    (["--L", "32", "--steps", "6", "--plan", "tblock,16,8,32,3"], 3),
])
def test_timing_cli_runs_the_requested_plan(argv, kernel, capsys):
    need_cuda()
    from paper_2309_10292_gb300 import timing
    timing.main(argv)
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert out["plan"]["kernel"] == kernel and out["gcups"] > 0
