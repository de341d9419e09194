"""The multi-GPU product function on one GPU: shard.energy_density_sharded run as two ranks
(two processes, gloo for the one gather of the coarse array) gives the E_c and coarse
densities of the single-process rpa_energy_density.  The ranks' kernels never wait on each
other, so sharing one GPU between them is safe; each rank runs only its own probe-points."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _opts():
    return dict(precision="fp64", lanczos_max=3, stern_tol=1e-10, stern_maxit=5000,
                stride=(2, 2, 2), interp="cubic")


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist

    import oracle
    import paper_2609_16408_gb300 as R
    from paper_2609_16408_gb300.shard import energy_density_sharded
    from tests.systems_small import small
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    s = small()
    om, w = oracle.gl_frequencies(3)
    c = R.Context.from_system(s, om, w, **_opts())
    P = R.rpa_num_probes(c.ctx)
    dco, ec = energy_density_sharded(c.ctx, P, len(om), s.N_d, rank, world,
                                     torch.device("cuda", 0))
    q.put((rank, dco.cpu().numpy(), float(ec)))
    c.close()
    dist.destroy_process_group()


def test_sharded_energy_equals_single_process():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp

    import oracle
    import paper_2609_16408_gb300 as R
    from tests.systems_small import small
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s = small()
    om, w = oracle.gl_frequencies(3)
    c = R.Context.from_system(s, om, w, **_opts())
    P = R.rpa_num_probes(c.ctx)
    dco, _, ec, _ = R.rpa_energy_density(c.ctx, len(om), P, s.N_d, want_fine=False)
    c.close()
    # the waves hold different probe-points in the two runs (and may pick different tilings),
    # so the solves agree to their tolerance (1e-10), not bit for bit
    for rank, d, e in res:
        assert np.allclose(d, dco, rtol=1e-9, atol=1e-14)
        assert abs(e - ec) <= 1e-9 * abs(ec)
