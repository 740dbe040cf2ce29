"""CUDA-graph capture of a step of libnbcore calls.

Every libnbcore entry point only enqueues kernels on the caller's stream: the list
rebuild is decided on the device (the rebuild kernels run on every step and return at
once unless the device-side flag is set), no call allocates or waits on the host, and
cuFFT executes under stream capture.  A whole step -- one force evaluation, or n
velocity-Verlet steps, of any number of batched systems -- can therefore be captured
once and replayed as a single graph launch, removing the per-kernel launch cost that
dominates small systems.
"""


class CapturedStep:
    """Capture ``fn`` (a callable issuing libnbcore calls on the current stream, with
    preallocated tensors) into a CUDA graph; ``replay()`` re-issues it.

    ``fn`` is run ``warmup`` times on a side stream first (the first call may build
    the list and lazily initialise library state), then captured.  Tensors that ``fn``
    reads or writes must stay alive and at the same addresses for the graph's lifetime.
    """

    def __init__(self, fn, warmup=2):
        import torch
        self._torch = torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            fn()

    def replay(self):
        self.graph.replay()
