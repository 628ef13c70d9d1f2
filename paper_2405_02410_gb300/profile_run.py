"""Run a fixed number of Model B steps for profilers (ncu wraps this command).

    python -m paper_2405_02410_gb300.profile_run --shape 1024 1024 --steps 20 [--eager] [--fields 1|2]
        [--tune key=value ...] [--adjoint] [--batch B] [--kpz]

--eager launches every step's kernels one by one (no CUDA graph); --fields 2
adds a Model A field (the 3D Model A + B pair); --tune passes launch-shape
settings to pss_set_tuning (e.g. fast2d=0 for the generic 2D kernels);
--adjoint runs the steps with checkpoints (pss_adjoint_forward) and then the
backward pass of J = |phi_T|^2 / 2 (pss_adjoint_backward) instead; --batch B
runs B independent 2D Model B instances in one batched system (seeds
2405 + i, the ensemble workload's parameters); --kpz runs the KPZ workload
(sigma 1, lambda 0.5, D 0.01) instead of Model B.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", type=int, nargs="+", default=[1024, 1024])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--fields", type=int, default=1)
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--eager", action="store_true")
    ap.add_argument("--tune", nargs="*", default=[], help="key=value launch-shape settings")
    ap.add_argument("--adjoint", action="store_true", help="forward with checkpoints, then the backward pass")
    ap.add_argument("--batch", type=int, default=1, help="independent 2D Model B instances in one batched system")
    ap.add_argument("--kpz", action="store_true", help="the KPZ workload instead of Model B")
    args = ap.parse_args()
    import torch
    from paper_2405_02410_gb300 import build
    build.build()
    from paper_2405_02410_gb300 import pss
    shape = tuple(args.shape)
    if len(shape) == 3:
        s = pss.System(shape, dt=0.005, seed=2405, precision=args.precision)
        if args.fields == 2:
            pss.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
        pss.add_model_b_field(s, a=-1, b=1, K=1, D=0.05, name="phi")
    elif args.kpz:
        s = pss.kpz(shape, dt=0.01, sigma=1.0, lam=0.5, D=0.01, seed=2405, precision=args.precision)
    elif args.batch > 1:
        s = pss.System(shape, dt=0.01, batch=args.batch, seeds=[2405 + i for i in range(args.batch)],
                       precision=args.precision)
        pss.add_model_b_field(s, a=-1.0, b=1.0, K=1.0, D=0.01)
    else:
        s = pss.model_b(shape, dt=0.01, a=-1, b=1, K=1, D=0.01, seed=2405, precision=args.precision)
        if args.fields == 2:
            pss.add_model_a_field(s, a=-1, b=1, K=1, D=0.05, name="psi")
    for kv in args.tune:
        k, v = kv.split("=")
        s.set_tuning(k, int(v))
    for b in range(args.batch):
        if args.batch > 1:
            s.select_instance(b)
        for f in range(args.fields):
            s.init_uniform(f, -0.1, 0.1)
    if args.adjoint:
        s.adjoint_forward(args.steps)
        s.adjoint_backward(s.get_spectrum(0), 4)
    elif args.eager:
        for _ in range(args.steps):
            s.step(1)
    else:
        s.step(args.steps)
    s.sync()
    torch.cuda.synchronize()
    print(f"ok: {shape} {args.steps} steps, launches={s.launch_count}")


if __name__ == "__main__":
    main()
