// The opaque handle behind the C ABI (shared by the .cu files of the ABI).
#pragma once

#include <memory>
#include <string>

#include "engine.cuh"

struct gbosqp_handle {
    gbosqp_settings s{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::unique_ptr<gb::EngineBase> eng;
    gbosqp_info info{};
    std::string err;
    double setup_ms = 0.0;
    long long setup_launches = 0;
};
