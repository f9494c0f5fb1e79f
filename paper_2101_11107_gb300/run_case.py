"""Run a named workload for a few steps on the GPU (for profiling and quick checks).

    python -m paper_2101_11107_gb300.run_case womersley fp32 4 [esoteric|ab] [launch config name]
    python -m paper_2101_11107_gb300.run_case aneurysm256 fp16 10
    python -m paper_2101_11107_gb300.run_case corrector128 fp32 50

Workloads: womersley (64x64x256 pulsatile pipe, radius 28), poiseuille (32x32x64 pipe,
radius 12), aneurysm256 / aneurysm512 (seeded synthetic aneurysm, seed 11); batch16: the 16
seeded aneurysms of the benchmark's batched variant (edges 96-192), advanced `steps` steps by one
batched launch per step (graph chunks of 10; launch config name as the last argument, or
"persistent"); corrector<edge>: the
learned corrector's forward pass (features, three convolutions, output) on the seed-200
synthetic aneurysm at that edge after 100 solver steps, repeated `steps` times (initial
parameters of seed 0), with its CUDA-event time per pass; corrector_train<edge>: the same case,
one training step per pass (forward, loss, backward with the weight gradients, Adam) toward a
seeded perturbation of u.
"""
import sys


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    case = argv[0] if argv else "womersley"
    storage = argv[1] if len(argv) > 1 else "fp32"
    steps = int(argv[2]) if len(argv) > 2 else 4
    scheme = argv[3] if len(argv) > 3 else "esoteric"
    config = argv[4] if len(argv) > 4 else None
    from . import build as lib_build
    from . import inputs as I
    from . import lbm

    lib_build.build()
    if case.startswith("corrector"):
        import torch

        train = case.startswith("corrector_train")
        edge = int(case[len("corrector_train" if train else "corrector"):] or 128)
        g = I.aneurysm(200, edge=edge, period=2000.0 * edge / 128.0)
        net = lbm.Corrector(g.mask, I.corrector_init_params(0), 0.05, 0.01, 0.005)
        dom = lbm.Domain.from_geometry(g)
        dom.step(100)
        rho, u = dom.macroscopic_tensors()
        u_target = u + 0.001 * torch.randn(u.shape, device=u.device, generator=torch.Generator(u.device).manual_seed(0))

        def one():
            if train:
                net.train_step(rho, u, u_target, 1e-4)
            else:
                net.forward(rho, u)

        for _ in range(3):
            one()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            one()
        e1.record()
        torch.cuda.synchronize()
        what = "train_step_ms" if train else "forward_ms"
        print(f"ok {case} fluid={g.nfluid} {what}={e0.elapsed_time(e1) / max(steps, 1):.4f}")
        return
    if case == "batch16":
        import numpy as np

        rng = np.random.default_rng(2024)
        edges = [int(96 + 16 * rng.integers(0, 7)) for _ in range(16)]
        doms = [lbm.Domain.from_geometry(I.aneurysm(300 + k, edge=e, wave_seed=400 + k), storage=storage)
                for k, e in enumerate(edges)]
        batch = lbm.Batch(doms, graph_steps=10)
        if config == "persistent":
            batch.set_persistent(True, 1.0)
        elif config is not None:
            batch.set_launch_config(lbm.LAUNCH_CONFIG_NAMES.index(config))
        batch.step(steps)
        batch.sync()
        print(f"ok batch16 {storage} steps={steps} fluid={batch.n_fluid} config={config}")
        batch.close()
        return
    if case == "womersley":
        g = I.womersley_pipe()
    elif case == "poiseuille":
        g = I.poiseuille_pipe_32()
    elif case.startswith("aneurysm"):
        g = I.aneurysm(11, edge=int(case[len("aneurysm"):] or 256))
    else:
        raise SystemExit(f"unknown case {case}")
    dom = lbm.Domain.from_geometry(g, storage=storage, scheme=scheme)
    if config is not None:
        dom.set_launch_config(lbm.LAUNCH_CONFIG_NAMES.index(config))
    dom.step(steps)
    dom.sync()
    info = dom.info()
    print(f"ok {case} {storage} {scheme} steps={steps} fluid={info['n_fluid']} slots={info['n_slots']} "
          f"config={lbm.LAUNCH_CONFIG_NAMES[info['launch_config']]}")


if __name__ == "__main__":
    main()
