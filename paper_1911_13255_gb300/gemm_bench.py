"""Time the tensor-core GEMM (sphfsi_gemm_bf16) at given shapes.

  python -m paper_1911_13255_gb300.gemm_bench [M N K] ...

Prints per shape the device time per call (CUDA events over 20 calls after 3
warm-up calls), the throughput and the error against FP32 products of the
same bfloat16 operands.  Default shapes: the learned sub-stepper's layer at a
training batch of 32 flag bodies (19 072 x 128 x 512), its weight gradient
(128 x 512 x 19 072) and a large square-ish product.
"""
import sys


def main(argv):
    import torch
    from . import gemm_bf16, tc_status

    vals = [int(v) for v in argv]
    shapes = [tuple(vals[i:i + 3]) for i in range(0, len(vals) - 2, 3)] or \
        [(19072, 128, 512), (128, 512, 19072), (16384, 256, 4096)]
    st = torch.cuda.Stream()
    for M, N, K in shapes:
        g = torch.Generator(device="cuda").manual_seed(M + N + K)
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        for _ in range(3):
            gemm_bf16(A, B, out=C, stream=st)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(20):
            gemm_bf16(A, B, out=C, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        ref = A.float() @ B.float().T
        err = ((C - ref).norm() / ref.norm()).item()
        print(f"M {M} N {N} K {K}: {ms * 1e3:.1f} us/call, {2.0 * M * N * K / ms / 1e9:.1f} TFLOP/s, "
              f"rel err {err:.2e}", flush=True)
    if tc_status():
        raise SystemExit("a bounded tensor-core wait ran out")


if __name__ == "__main__":
    main(sys.argv[1:])
