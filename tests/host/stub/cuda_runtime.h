/* Empty stand-in for the CUDA runtime header: the host unit test of the
 * double-float header needs none of its declarations. */
#pragma once
