"""The handle's device footprint (isc_get_device_bytes): every allocation is
counted (the device's free memory drops by the reported bytes, up to the
allocator's rounding), the arrays made at creation come to the FP64 layout's
per-cell size with GMRES(30), the mixed modes' FP32 copies are added on their
first use, and closing the handle returns all of it."""
import pytest

import isc_inputs as inp

pytestmark = pytest.mark.gpu


def test_device_bytes_match_free_memory_and_the_layout():
    torch = pytest.importorskip("torch")
    from paper_1811_11992_gb300 import build
    build.build()
    from paper_1811_11992_gb300 import Simulator

    # load the library's kernels first (module code and static data are not the handle's)
    w = Simulator(inp.small_box(4, 3, 2))
    w.init_equilibrium()
    w.newton_step(60.0)
    w.set_options(precision="mixed_fgmres")
    w.newton_step(60.0)
    w.close()
    torch.cuda.synchronize()

    case = inp.config(3)                       # 100x100x30, 300,000 cells
    n, (nx, ny, nz) = case.n, (case.nx, case.ny, case.nz)
    nnzb = 7 * n - 2 * (ny * nz + nx * nz + nx * ny)
    free0 = torch.cuda.mem_get_info()[0]
    g = Simulator(case, tol_lin=1e-6)
    nb = g.device_bytes()
    free1 = torch.cuda.mem_get_info()[0]
    slack = 64 * 2**21                         # 2 MiB rounding on up to 64 allocations
    assert nb - 2**22 <= free0 - free1 <= nb + slack
    # Jacobian blocks, 61 GMRES vectors, D^-1 and three upper blocks, staged face quantities
    assert nb >= nnzb * 512 + 61 * 8 * n * 8 + 4 * 512 * n + 1152 * n
    assert nb / n < 12_000

    # the FP32 preconditioner copies and the inner basis come with the first mixed solve
    g.init_equilibrium()
    g.set_options(precision="mixed_fgmres")
    g.newton_step(case.dt0)
    nb2 = g.device_bytes()
    inner = g.options.inner_its
    assert nb2 - nb >= nnzb * 256 + 4 * 256 * n + (2 * inner + 2) * 8 * n * 4
    free2 = torch.cuda.mem_get_info()[0]
    assert nb2 - 2**22 <= free0 - free2 <= nb2 + slack

    g.close()
    free3 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free3) <= slack
